/*
 * ADMM iterations of the paper for the oracle (TEST INFRASTRUCTURE ONLY).
 *
 *  - Algorithm 2 (OD2P_m, section 3.1): nonblind, D >= 1 subdomains.  With
 *    D = 2 it is Algorithm 1 (OD2P, section 2.3); with D = 1 it is ADMM on the
 *    whole domain.
 *  - Algorithm 3 (OD2BP, section 3.2): blind, the probe is recovered too.
 *
 * Steps are taken in the paper's order and notation.  Readings of points the
 * paper leaves open:
 *  - Step 1 uses lambda = eta in the ST-AGM prox (eq. updateZ).
 *  - Pairs: every ordered pair (d, e) whose rectangles intersect has its own
 *    multiplier Lambda_{d,e} on Omega_d n Omega_e; v_{d,e} = v_{e,d}
 *    (eq. updateV-multi).  The Step 3 diagonal pi^T pi sums to c_d(p), the
 *    number of other subdomains containing p.
 *  - Step 3 closed form (eq. Alg1-solver-u and its D-subdomain analogue):
 *      u = (eta A_d^*(z - Gamma) + r sum_e (v_{d,e} - Lambda_{d,e}))
 *          / (eta sum_j S_j^T |w|^2 + r c_d);
 *    a pixel whose denominator is exactly 0 (no illumination, no overlap)
 *    keeps its value (the paper fixes such boundary pixels, section 4).
 *  - Blind: the w-update averages the D copies, w = (1/D) F^* M F sum_d(Delta_d
 *    + W_d) (eq. blind_w has 1/2 for D = 2); M is 1 on the Fourier support of
 *    the probe and 0 on the zero set (the paper's definition of M has the two
 *    swapped); D_U^* D_U is sum_j |S_j u_d|^2 (eq. blind_W); the U-update has
 *    the proximal weight gamma (eq. blind_U).
 *  - RF (section 4) is accumulated from the frames A_d u_d^n (blind:
 *    F(W_d^n o S_j u_d^n)) formed in Step 1, i.e. it is the RF of the iterate
 *    entering the iteration.  RE = max_d ||u_d^{n+1} - u_d^n|| / ||u_d^{n+1}||.
 *  - Periodic boundaries (the torus reading in geometry.c): windows are read
 *    at the frames' placed offsets in extended coordinates; pair k = (d, e, s)
 *    couples pixel (R, C) of u_d with pixel (R - s_r H, C - s_c W) of u_e, and
 *    Lambda_{e,d} is read at that pixel of the reverse pair (e, d, -s); v uses
 *    the operand order of the pair listed first (d < e, or d = e with the
 *    positive shift).  Step 0 reads u0 modulo the image; the merge averages
 *    every copy of an image pixel.  Without periodic boundaries every shift is
 *    0 and these are the steps above, operation for operation.
 *  - Subdomain ownership (section 3.1: the subdomains are independent but for
 *    the overlap terms): with an ownership mask set, an iteration updates only
 *    the owned subdomains -- their frames, u_d, Lambda_{d,e}, and (blind) W_d
 *    and Delta_d -- and reads the other subdomains' u_e, Lambda_{e,d}, W_e and
 *    Delta_e as they were last set (their halo copies).  RF and RE then cover
 *    the owned part only.  Every owned value is computed exactly as without a
 *    mask, so ranks that own disjoint sets and exchange those copies between
 *    iterations reproduce the undivided iteration.
 */
#include "od2p_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

struct orc_admm {
    int H, W, m, mm, J, D, P, blind, periodic;
    int32_t *offs, *frame_sub, *rect, *pair, *pair_shift, *pair_rect;
    int *rev, *first;      /* P: index of the reverse pair (e, d, -s); 1 for the pair listed first */
    int *pd_begin;         /* D + 1: pairs of subdomain d are [pd_begin[d], pd_begin[d + 1]) */
    double eps, eta, r, mu, gamma;
    double *f, *mask;      /* J*mm, mm */
    ocplx *w, *Wd, *Delta; /* mm, D*mm, D*mm */
    ocplx *u, *Gamma, *Lam, *v, *z;
    int64_t *u_off, *lam_off;
    int32_t *owned;        /* D: 1 where this instance updates subdomain d */
    double rf, re;
};

static inline int wrapi(int x, int n) { int r = x % n; return r < 0 ? r + n : r; }
static inline int rh(const int32_t *rc) { return rc[2] - rc[0]; }
static inline int rw(const int32_t *rc) { return rc[3] - rc[1]; }

/* index of global pixel (R, C) inside rectangle rc, or -1 */
static inline int64_t rect_idx(const int32_t *rc, int R, int C)
{
    if (R < rc[0] || R >= rc[2] || C < rc[1] || C >= rc[3]) return -1;
    return (int64_t)(R - rc[0]) * rw(rc) + (C - rc[1]);
}

orc_admm *orc_admm_new_ext(int H, int W, int m, int J, const int32_t *offs, int sub_rows,
                           int sub_cols, int overlap_px, int periodic, const double *f, const ocplx *w0,
                           const ocplx *u0, double eps, double eta, double r, int blind,
                           double mu, double gamma, const double *mask)
{
    orc_admm *s = (orc_admm *)calloc(1, sizeof(orc_admm));
    s->H = H; s->W = W; s->m = m; s->mm = m * m; s->J = J; s->blind = blind; s->periodic = periodic != 0;
    s->eps = eps; s->eta = eta; s->r = r; s->mu = mu; s->gamma = gamma;
    const int mm = s->mm, D0 = sub_rows * sub_cols;
    /* offs holds each frame's placed offset (extended coordinates; the given offset when not periodic) */
    s->offs = (int32_t *)malloc(sizeof(int32_t) * 2 * (J > 0 ? J : 1));
    s->frame_sub = (int32_t *)malloc(sizeof(int32_t) * (J > 0 ? J : 1));
    s->rect = (int32_t *)malloc(sizeof(int32_t) * 4 * D0);
    s->D = orc_geometry_ext(H, W, m, J, offs, sub_rows, sub_cols, overlap_px, s->periodic, s->frame_sub, s->rect,
                            s->offs);
    if (s->D <= 0) { free(s->offs); free(s->frame_sub); free(s->rect); free(s); return NULL; }
    const int D = s->D;
    s->P = orc_pairs_ext(D, s->rect, H, W, s->periodic, 0, NULL, NULL, NULL);
    s->pair = (int32_t *)malloc(sizeof(int32_t) * 2 * (s->P + 1));
    s->pair_shift = (int32_t *)malloc(sizeof(int32_t) * 2 * (s->P + 1));
    s->pair_rect = (int32_t *)malloc(sizeof(int32_t) * 4 * (s->P + 1));
    orc_pairs_ext(D, s->rect, H, W, s->periodic, s->P, s->pair, s->pair_shift, s->pair_rect);
    s->rev = (int *)malloc(sizeof(int) * (s->P + 1));
    s->first = (int *)malloc(sizeof(int) * (s->P + 1));
    for (int k = 0; k < s->P; ++k) {
        const int d = s->pair[2 * k], e = s->pair[2 * k + 1], sr = s->pair_shift[2 * k], sc = s->pair_shift[2 * k + 1];
        s->rev[k] = -1;
        for (int q = 0; q < s->P; ++q)
            if (s->pair[2 * q] == e && s->pair[2 * q + 1] == d && s->pair_shift[2 * q] == -sr &&
                s->pair_shift[2 * q + 1] == -sc)
                s->rev[k] = q;
        s->first[k] = d < e || (d == e && (sr > 0 || (sr == 0 && sc > 0)));
    }
    s->pd_begin = (int *)malloc(sizeof(int) * (D + 1));
    for (int d = 0, k = 0; d <= D; ++d) {
        while (k < s->P && s->pair[2 * k] < d) ++k;
        s->pd_begin[d] = k;
    }

    s->u_off = (int64_t *)malloc(sizeof(int64_t) * (D + 1));
    s->u_off[0] = 0;
    for (int d = 0; d < D; ++d) s->u_off[d + 1] = s->u_off[d] + (int64_t)rh(s->rect + 4 * d) * rw(s->rect + 4 * d);
    s->lam_off = (int64_t *)malloc(sizeof(int64_t) * (s->P + 1));
    s->lam_off[0] = 0;
    for (int k = 0; k < s->P; ++k)
        s->lam_off[k + 1] = s->lam_off[k] + (int64_t)rh(s->pair_rect + 4 * k) * rw(s->pair_rect + 4 * k);

    s->f = (double *)malloc(sizeof(double) * (size_t)J * mm + 1);
    memcpy(s->f, f, sizeof(double) * (size_t)J * mm);
    s->mask = (double *)malloc(sizeof(double) * mm);
    for (int k = 0; k < mm; ++k) s->mask[k] = mask ? mask[k] : 1.0;
    s->w = (ocplx *)malloc(sizeof(ocplx) * mm);
    memcpy(s->w, w0, sizeof(ocplx) * mm);
    s->Wd = (ocplx *)malloc(sizeof(ocplx) * (size_t)D * mm);
    s->Delta = (ocplx *)calloc((size_t)D * mm, sizeof(ocplx));
    for (int d = 0; d < D; ++d) memcpy(s->Wd + (size_t)d * mm, w0, sizeof(ocplx) * mm);

    /* Step 0: u_d^0 = R_d u0 (ones when u0 is NULL), Gamma^0 = Lambda^0 = 0 */
    s->u = (ocplx *)malloc(sizeof(ocplx) * (size_t)s->u_off[D]);
    for (int d = 0; d < D; ++d) {
        const int32_t *rc = s->rect + 4 * d;
        for (int R = rc[0]; R < rc[2]; ++R)
            for (int C = rc[1]; C < rc[3]; ++C)
                s->u[s->u_off[d] + rect_idx(rc, R, C)] = u0 ? u0[(size_t)wrapi(R, H) * W + wrapi(C, W)] : 1.0;
    }
    s->Gamma = (ocplx *)calloc((size_t)J * mm + 1, sizeof(ocplx));
    s->z = (ocplx *)calloc((size_t)J * mm + 1, sizeof(ocplx));
    s->Lam = (ocplx *)calloc((size_t)s->lam_off[s->P] + 1, sizeof(ocplx));
    s->v = (ocplx *)calloc((size_t)s->lam_off[s->P] + 1, sizeof(ocplx));
    s->owned = (int32_t *)malloc(sizeof(int32_t) * D);
    for (int d = 0; d < D; ++d) s->owned[d] = 1;
    return s;
}

void orc_admm_set_owned(orc_admm *s, const int32_t *owned)
{
    for (int d = 0; d < s->D; ++d) s->owned[d] = owned ? (owned[d] != 0) : 1;
}

void orc_admm_free(orc_admm *s)
{
    if (!s) return;
    free(s->offs); free(s->frame_sub); free(s->rect); free(s->pair); free(s->pair_shift); free(s->pair_rect);
    free(s->rev); free(s->first); free(s->pd_begin); free(s->f); free(s->mask); free(s->w); free(s->Wd); free(s->Delta);
    free(s->u); free(s->Gamma); free(s->Lam); free(s->v); free(s->z); free(s->u_off);
    free(s->lam_off); free(s->owned); free(s);
}

int orc_admm_num_sub(const orc_admm *s) { return s->D; }
int orc_admm_num_pairs(const orc_admm *s) { return s->P; }

static inline ocplx *u_at(orc_admm *s, int d, int R, int C)
{
    int64_t i = rect_idx(s->rect + 4 * d, R, C);
    return i < 0 ? NULL : s->u + s->u_off[d] + i;
}

static inline ocplx *lam_at(ocplx *base, const orc_admm *s, int k, int R, int C)
{
    return base + s->lam_off[k] + rect_idx(s->pair_rect + 4 * k, R, C);
}

void orc_admm_iterate(orc_admm *s, int n_iter)
{
    const int m = s->m, mm = s->mm, J = s->J, D = s->D;
    ocplx *X = (ocplx *)malloc(sizeof(ocplx) * (size_t)J * mm + 1);
    ocplx *Q = (ocplx *)malloc(sizeof(ocplx) * (size_t)J * mm + 1);
    ocplx *unew = (ocplx *)malloc(sizeof(ocplx) * (size_t)s->u_off[D] + 1);
    ocplx *acc = (ocplx *)malloc(sizeof(ocplx) * (size_t)s->u_off[D] + 1);
    double *nrm = (double *)malloc(sizeof(double) * (size_t)s->u_off[D] + 1);
    ocplx *wnew = (ocplx *)malloc(sizeof(ocplx) * mm);
    ocplx *Wnew = (ocplx *)malloc(sizeof(ocplx) * (size_t)D * mm);
    double *rfj = (double *)malloc(sizeof(double) * (J + 1));

    for (int it = 0; it < n_iter; ++it) {
        /* ---------------- Step 1 ---------------- */
        if (s->blind) { /* w^{n+1} = (1/D) F^* M F sum_d (Delta_d^n + W_d^n)   (eq. blind_w) */
            for (int k = 0; k < mm; ++k) {
                ocplx t = 0.0;
                for (int d = 0; d < D; ++d) t += s->Delta[(size_t)d * mm + k] + s->Wd[(size_t)d * mm + k];
                wnew[k] = t;
            }
            orc_fft2(wnew, m, 0);
            for (int k = 0; k < mm; ++k) wnew[k] *= s->mask[k];
            orc_fft2(wnew, m, 1);
            for (int k = 0; k < mm; ++k) wnew[k] /= (double)D;
        }
        /* z_d^{n+1} = Prox_{G_eps; eta}(Gamma_d^n + A_d u_d^n)           (eq. updateZ / blind_Z) */
#pragma omp parallel for schedule(static)
        for (int j = 0; j < J; ++j) {
            const int d = s->frame_sub[j];
            rfj[j] = 0.0;
            if (!s->owned[d]) continue;
            const ocplx *wp = s->blind ? s->Wd + (size_t)d * mm : s->w;
            ocplx *x = X + (size_t)j * mm;
            const int r0 = s->offs[2 * j], c0 = s->offs[2 * j + 1];
            for (int r = 0; r < m; ++r)
                for (int c = 0; c < m; ++c)
                    x[r * m + c] = wp[r * m + c] * *u_at(s, d, r0 + r, c0 + c);
            orc_fft2(x, m, 0);
            double rs = 0.0;
            for (int k = 0; k < mm; ++k) {
                const double fk = s->f[(size_t)j * mm + k];
                rs += fabs(cabs(x[k]) - sqrt(fk));
                s->z[(size_t)j * mm + k] = orc_stagm_prox(s->Gamma[(size_t)j * mm + k] + x[k], fk, s->eps, s->eta);
            }
            rfj[j] = rs;
        }
        {
            double num = 0.0, den = 0.0;
            for (int j = 0; j < J; ++j) num += rfj[j];
            for (int j = 0; j < J; ++j)
                if (s->owned[s->frame_sub[j]])
                    for (int k = 0; k < mm; ++k) den += sqrt(s->f[(size_t)j * mm + k]);
            s->rf = den > 0.0 ? num / den : 0.0;
        }
        /* v_{i1,i2}^{n+1} = 1/2 (pi u_i1^n + pi u_i2^n + Lambda_{i1,i2}^n + Lambda_{i2,i1}^n) (eq. updateV-multi) */
        for (int k = 0; k < s->P; ++k) {
            const int d = s->pair[2 * k], e = s->pair[2 * k + 1], kr = s->rev[k];
            if (!s->owned[d]) continue;
            const int sR = s->pair_shift[2 * k] * s->H, sC = s->pair_shift[2 * k + 1] * s->W;
            const int32_t *prc = s->pair_rect + 4 * k;
            for (int R = prc[0]; R < prc[2]; ++R)
                for (int C = prc[1]; C < prc[3]; ++C) {
                    const ocplx ud = *u_at(s, d, R, C), ue = *u_at(s, e, R - sR, C - sC);
                    const ocplx ld = *lam_at(s->Lam, s, k, R, C), le = *lam_at(s->Lam, s, kr, R - sR, C - sC);
                    *lam_at(s->v, s, k, R, C) = s->first[k] ? 0.5 * (ud + ue + ld + le) : 0.5 * (ue + ud + le + ld);
                }
        }
        /* ---------------- Step 2: Gamma^{n+1} = Gamma^n + A_d u_d^n - z^{n+1}  (eq. updateM-1-multi) */
        for (int j = 0; j < J; ++j)
            if (s->owned[s->frame_sub[j]])
                for (int k = 0; k < mm; ++k) s->Gamma[(size_t)j * mm + k] += X[(size_t)j * mm + k] - s->z[(size_t)j * mm + k];

        /* q_j = F^*(z_j - Gamma_j^{n+1}) (shared by the blind W- and U-updates and A_d^*) */
#pragma omp parallel for schedule(static)
        for (int j = 0; j < J; ++j) {
            if (!s->owned[s->frame_sub[j]]) continue;
            ocplx *q = Q + (size_t)j * mm;
            for (int k = 0; k < mm; ++k) q[k] = s->z[(size_t)j * mm + k] - s->Gamma[(size_t)j * mm + k];
            orc_fft2(q, m, 1);
        }

        /* ---------------- Step 3 (blind): W-update, eq. blind_W, uses u^n */
        if (s->blind) {
            for (int d = 0; d < D; ++d) {
                ocplx *Wn = Wnew + (size_t)d * mm;
                if (!s->owned[d]) {  /* another instance's subdomain: keep its copy */
                    memcpy(Wn, s->Wd + (size_t)d * mm, sizeof(ocplx) * mm);
                    continue;
                }
                double *dd = (double *)calloc(mm, sizeof(double));
                for (int k = 0; k < mm; ++k) Wn[k] = 0.0;
                for (int j = 0; j < J; ++j) {
                    if (s->frame_sub[j] != d) continue;
                    const int r0 = s->offs[2 * j], c0 = s->offs[2 * j + 1];
                    for (int r = 0; r < m; ++r)
                        for (int c = 0; c < m; ++c) {
                            ocplx uu = *u_at(s, d, r0 + r, c0 + c);
                            Wn[r * m + c] += conj(uu) * Q[(size_t)j * mm + r * m + c];
                            dd[r * m + c] += creal(uu) * creal(uu) + cimag(uu) * cimag(uu);
                        }
                }
                for (int k = 0; k < mm; ++k)
                    Wn[k] = (s->eta * Wn[k] + s->mu * (wnew[k] - s->Delta[(size_t)d * mm + k])) /
                            (s->eta * dd[k] + s->mu);
                free(dd);
            }
        }

        /* ---------------- Step 3 (nonblind) / Step 4 (blind): u-update */
        const ocplx *Wuse = s->blind ? Wnew : NULL;
        memset(acc, 0, sizeof(ocplx) * (size_t)s->u_off[D]);
        memset(nrm, 0, sizeof(double) * (size_t)s->u_off[D]);
        for (int j = 0; j < J; ++j) {
            const int d = s->frame_sub[j];
            if (!s->owned[d]) continue;
            const ocplx *wp = Wuse ? Wuse + (size_t)d * mm : s->w;
            const int r0 = s->offs[2 * j], c0 = s->offs[2 * j + 1];
            for (int r = 0; r < m; ++r)
                for (int c = 0; c < m; ++c) {
                    int64_t i = s->u_off[d] + rect_idx(s->rect + 4 * d, r0 + r, c0 + c);
                    ocplx wk = wp[r * m + c];
                    acc[i] += conj(wk) * Q[(size_t)j * mm + r * m + c];
                    nrm[i] += creal(wk) * creal(wk) + cimag(wk) * cimag(wk);
                }
        }
        s->re = 0.0;
        for (int d = 0; d < D; ++d) {
            const int32_t *rc = s->rect + 4 * d;
            if (!s->owned[d]) {  /* another instance's subdomain: keep its copy */
                memcpy(unew + s->u_off[d], s->u + s->u_off[d], sizeof(ocplx) * (size_t)(s->u_off[d + 1] - s->u_off[d]));
                continue;
            }
            double dn = 0.0, nn = 0.0;
            for (int R = rc[0]; R < rc[2]; ++R)
                for (int C = rc[1]; C < rc[3]; ++C) {
                    int64_t i = s->u_off[d] + rect_idx(rc, R, C);
                    ocplx num = s->eta * acc[i];
                    double den = s->eta * nrm[i];
                    for (int k = s->pd_begin[d]; k < s->pd_begin[d + 1]; ++k) {
                        if (rect_idx(s->pair_rect + 4 * k, R, C) < 0) continue;
                        num += s->r * (*lam_at(s->v, s, k, R, C) - *lam_at(s->Lam, s, k, R, C));
                        den += s->r;
                    }
                    if (s->blind) {
                        num += s->gamma * s->u[i];
                        den += s->gamma;
                    }
                    unew[i] = den > 0.0 ? num / den : s->u[i];
                    ocplx dlt = unew[i] - s->u[i];
                    dn += creal(dlt) * creal(dlt) + cimag(dlt) * cimag(dlt);
                    nn += creal(unew[i]) * creal(unew[i]) + cimag(unew[i]) * cimag(unew[i]);
                }
            double red = nn > 0.0 ? sqrt(dn / nn) : 0.0;
            if (red > s->re) s->re = red;
        }
        memcpy(s->u, unew, sizeof(ocplx) * (size_t)s->u_off[D]);

        /* ---------------- Step 4 / Step 5: multipliers (eqs. updateM-2-multi, admm_Delta, admm_Lambda) */
        if (s->blind) {
            for (int d = 0; d < D; ++d) {
                if (!s->owned[d]) continue;
                for (int k = 0; k < mm; ++k) {
                    s->Delta[(size_t)d * mm + k] += Wnew[(size_t)d * mm + k] - wnew[k];
                    s->Wd[(size_t)d * mm + k] = Wnew[(size_t)d * mm + k];
                }
            }
            memcpy(s->w, wnew, sizeof(ocplx) * mm);
        }
        for (int k = 0; k < s->P; ++k) {
            const int d = s->pair[2 * k];
            if (!s->owned[d]) continue;
            const int32_t *prc = s->pair_rect + 4 * k;
            for (int R = prc[0]; R < prc[2]; ++R)
                for (int C = prc[1]; C < prc[3]; ++C)
                    *lam_at(s->Lam, s, k, R, C) += *u_at(s, d, R, C) - *lam_at(s->v, s, k, R, C);
        }
    }
    free(X); free(Q); free(unew); free(acc); free(nrm); free(wnew); free(Wnew); free(rfj);
}

int64_t orc_admm_state_len(const orc_admm *s, int which)
{
    switch (which) {
    case 0: return s->u_off[s->D];
    case 1: case 7: return (int64_t)s->J * s->mm;
    case 2: case 6: return s->lam_off[s->P];
    case 3: case 4: return (int64_t)s->D * s->mm;
    case 5: return s->mm;
    default: return -1;
    }
}

static ocplx *state_ptr(const orc_admm *s, int which)
{
    switch (which) {
    case 0: return s->u;
    case 1: return s->Gamma;
    case 2: return s->Lam;
    case 3: return s->Wd;
    case 4: return s->Delta;
    case 5: return s->w;
    case 6: return s->v;
    case 7: return s->z;
    default: return NULL;
    }
}

void orc_admm_get(const orc_admm *s, int which, ocplx *out)
{
    int64_t n = orc_admm_state_len(s, which);
    if (n > 0) memcpy(out, state_ptr(s, which), sizeof(ocplx) * (size_t)n);
}

void orc_admm_set(orc_admm *s, int which, const ocplx *in)
{
    int64_t n = orc_admm_state_len(s, which);
    if (n > 0) memcpy(state_ptr(s, which), in, sizeof(ocplx) * (size_t)n);
}

void orc_admm_metrics(const orc_admm *s, double *rf, double *re)
{
    if (rf) *rf = s->rf;
    if (re) *re = s->re;
}

/* Section 4 set-up: non-overlapping pixels keep their value, overlaps are averaged. */
void orc_admm_merge(const orc_admm *s, ocplx *u_out)
{
    const int smax = s->periodic ? 2 : 0;
    for (int R = 0; R < s->H; ++R)
        for (int C = 0; C < s->W; ++C) {
            ocplx t = 0.0;
            int n = 0;
            for (int d = 0; d < s->D; ++d)
                for (int sr = -smax; sr <= smax; ++sr)
                    for (int sc = -smax; sc <= smax; ++sc) {
                        int64_t i = rect_idx(s->rect + 4 * d, R + sr * s->H, C + sc * s->W);
                        if (i < 0) continue;
                        t += s->u[s->u_off[d] + i];
                        ++n;
                    }
            u_out[(size_t)R * s->W + C] = n ? t / (double)n : 1.0;
        }
}

/* Change the penalties eta (z = A u splitting) and r (v = pi u consensus)
 * between iterations.  Gamma and Lambda are the scaled multipliers of the
 * augmented Lagrangian, so the unscaled ones (eta Gamma, r Lambda) are kept:
 * Gamma <- (eta / eta') Gamma, Lambda <- (r / r') Lambda (the rescaling of
 * Boyd, Parikh, Chu, Peleato, Eckstein 2011, section 3.4.1).                */
void orc_admm_set_penalties(orc_admm *s, double eta, double r)
{
    const double ge = s->eta / eta;
    for (int64_t k = 0; k < (int64_t)s->J * s->mm; ++k) s->Gamma[k] *= ge;
    if (r > 0.0) {
        const double gl = s->r / r;
        for (int64_t k = 0; k < s->lam_off[s->P]; ++k) s->Lam[k] *= gl;
    }
    s->eta = eta;
    s->r = r;
}

/* Consensus residual: || u_d - u_e || over every ordered pair's overlap,
 * relative to || u || over all subdomain pixels (0 when there are no pairs). */
double orc_admm_consensus(const orc_admm *s)
{
    double num = 0.0, den = 0.0;
    for (int k = 0; k < s->P; ++k) {
        const int d = s->pair[2 * k], e = s->pair[2 * k + 1];
        const int sR = s->pair_shift[2 * k] * s->H, sC = s->pair_shift[2 * k + 1] * s->W;
        const int32_t *pr = s->pair_rect + 4 * k;
        for (int R = pr[0]; R < pr[2]; ++R)
            for (int C = pr[1]; C < pr[3]; ++C) {
                const ocplx a = s->u[s->u_off[d] + rect_idx(s->rect + 4 * d, R, C)];
                const ocplx b = s->u[s->u_off[e] + rect_idx(s->rect + 4 * e, R - sR, C - sC)];
                const ocplx t = a - b;
                num += creal(t) * creal(t) + cimag(t) * cimag(t);
            }
    }
    for (int64_t k = 0; k < s->u_off[s->D]; ++k) den += creal(s->u[k]) * creal(s->u[k]) + cimag(s->u[k]) * cimag(s->u[k]);
    return den > 0.0 ? sqrt(num / den) : 0.0;
}

orc_admm *orc_admm_new(int H, int W, int m, int J, const int32_t *offs, int sub_rows,
                       int sub_cols, int overlap_px, const double *f, const ocplx *w0,
                       const ocplx *u0, double eps, double eta, double r, int blind,
                       double mu, double gamma, const double *mask)
{
    return orc_admm_new_ext(H, W, m, J, offs, sub_rows, sub_cols, overlap_px, 0, f, w0, u0, eps, eta, r, blind, mu,
                            gamma, mask);
}
