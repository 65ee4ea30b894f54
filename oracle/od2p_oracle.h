/*
 * FP64 CPU oracle for the OD2P / OD2P_m / OD2BP ptychography iteration of
 * Chang, Glowinski, Marchesini, Tai, Wang, Zeng, "Overlapping Domain
 * Decomposition Methods for Ptychographic Imaging" (arXiv:2011.00162).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no code, header, table
 * or helper with the CUDA library; every routine below is written from the
 * paper's definitions in double precision (C99 `double complex`).
 *
 * Complex arrays are interleaved (re, im) doubles, i.e. `double complex`.
 * Images and frames are row-major.  The DFT is unitary (1/sqrt(N) both ways)
 * and returns frequencies in natural (unshifted) order.
 */
#ifndef OD2P_ORACLE_H
#define OD2P_ORACLE_H

#include <complex.h>
#include <stdint.h>

typedef double complex ocplx;

#define ORC_PI 3.14159265358979323846264338327950288

/* ---- unitary 2-D DFT (section 2: "normalized discrete Fourier transform") ---- */
void orc_dft2(ocplx *x, int m, int inverse);   /* naive O(m^4) definition    */
void orc_fft2(ocplx *x, int m, int inverse);   /* radix-2 (m = 2^k), else row/column definition */

/* ---- ST-AGM, section 2.2 ---- */
double orc_stagm_g(ocplx x, double b, double eps);                  /* eq. (obj-1)    */
ocplx  orc_stagm_grad(ocplx x, double b, double eps);               /* eq. (objgrad)  */
ocplx  orc_stagm_prox(ocplx y, double f, double eps, double lam);   /* eq. (Prox_sol) */
void orc_stagm_g_arr(const ocplx *x, const double *b, int64_t n, double eps, double *out);
void orc_stagm_grad_arr(const ocplx *x, const double *b, int64_t n, double eps, ocplx *out);
void orc_stagm_prox_arr(const ocplx *y, const double *f, int64_t n, double eps, double lam,
                        ocplx *z);

/* ---- forward operator A and its adjoint, section 2 (problem PtychoPR) ---- */
/* out[j] = F(w o S_j u) for all J frames; offs is J x 2 (row, col).           */
void orc_forward(int H, int W, const ocplx *u, int m, const ocplx *w, int J,
                 const int32_t *offs, ocplx *out);
/* u_out = A^* y = sum_j S_j^T (conj(w) o F^* y_j)   (H x W, overwritten).       */
void orc_adjoint(int H, int W, int m, const ocplx *w, int J, const int32_t *offs,
                 const ocplx *y, ocplx *u_out);
/* ST-AGM data-fidelity loss sum_j G_eps(F(w o S_j u); f_j) and its gradients
 * (d/dRe + i d/dIm) w.r.t. u (H x W) and w (m x m); either gradient may be NULL. */
double orc_loss_grad(int H, int W, const ocplx *u, int m, const ocplx *w, int J,
                     const int32_t *offs, const double *f, double eps, ocplx *gu, ocplx *gw);
/* The same with periodic != 0: windows wrap modulo H x W (geometry.c's torus reading). */
void orc_forward_ext(int H, int W, const ocplx *u, int m, const ocplx *w, int J,
                     const int32_t *offs, int periodic, ocplx *out);
void orc_adjoint_ext(int H, int W, int m, const ocplx *w, int J, const int32_t *offs, int periodic,
                     const ocplx *y, ocplx *u_out);
double orc_loss_grad_ext(int H, int W, const ocplx *u, int m, const ocplx *w, int J,
                         const int32_t *offs, int periodic, const double *f, double eps, ocplx *gu, ocplx *gw);

/* Data-driven initial probe of the blind experiments (section 4.2): the mean
 * over the J frames of the inverse unitary DFT of the measured amplitudes,
 * w0 = (1/J) sum_j F^* sqrt(f_j), taken frame by frame.  f: J x m x m.       */
void orc_probe_init(int m, int J, const double *f, ocplx *w0);

/* Section 4's SNR in dB of u_g against u_r after global-phase alignment. */
double orc_snr(int64_t n, const ocplx *ur, const ocplx *ug);

/* ---- overlapping domain decomposition, sections 2.1 and 3.1 ---- */
/* frame_sub[J]: subdomain of each frame; rect[D*4]: (r0, c0, r1, c1) half-open.
 * Returns D (= sub_rows*sub_cols) or a negative value on invalid input.        */
int orc_geometry(int H, int W, int m, int J, const int32_t *offs, int sub_rows,
                 int sub_cols, int overlap_px, int32_t *frame_sub, int32_t *rect);
/* Ordered pairs (d, e), d != e, whose rectangles intersect, sorted by (d, e).
 * pair[k*2..], pair_rect[k*4..]; returns the number of pairs (<= max_pairs).   */
int orc_pairs(int D, const int32_t *rect, int max_pairs, int32_t *pair, int32_t *pair_rect);
/* Either variant (periodic != 0: the torus reading in geometry.c).  roffs[J*2]
 * (may be NULL): each frame's offset in extended coordinates.  Pairs (d, e, s)
 * sorted by (d, e, s_r, s_c), s in {-2, ..., 2}^2 (only 0 when not periodic);
 * pair_shift[k*2..] = s (may be NULL); pair_rect in d's coordinates.  -3: a
 * rectangle reaching outside (-H, 2H) x (-W, 2W).                              */
int orc_geometry_ext(int H, int W, int m, int J, const int32_t *offs, int sub_rows, int sub_cols,
                     int overlap_px, int periodic, int32_t *frame_sub, int32_t *rect, int32_t *roffs);
int orc_pairs_ext(int D, const int32_t *rect, int H, int W, int periodic, int max_pairs, int32_t *pair,
                  int32_t *pair_shift, int32_t *pair_rect);

/* ---- ADMM state: Algorithm 2 (OD2P_m, nonblind) and Algorithm 3 (OD2BP) ---- */
typedef struct orc_admm orc_admm;

/* f: J x m x m measured intensities.  w0: initial (nonblind: known) probe.
 * u0: initial full image H x W or NULL for all ones (Step 0).  mask: m x m
 * Fourier support of the probe (1 on the support) or NULL for all ones.       */
orc_admm *orc_admm_new(int H, int W, int m, int J, const int32_t *offs, int sub_rows,
                       int sub_cols, int overlap_px, const double *f, const ocplx *w0,
                       const ocplx *u0, double eps, double eta, double r, int blind,
                       double mu, double gamma, const double *mask);
/* Either boundary variant (periodic != 0: the torus reading in geometry.c). */
orc_admm *orc_admm_new_ext(int H, int W, int m, int J, const int32_t *offs, int sub_rows,
                           int sub_cols, int overlap_px, int periodic, const double *f, const ocplx *w0,
                           const ocplx *u0, double eps, double eta, double r, int blind,
                           double mu, double gamma, const double *mask);
void orc_admm_free(orc_admm *s);
void orc_admm_iterate(orc_admm *s, int n_iter);
int  orc_admm_num_sub(const orc_admm *s);
int  orc_admm_num_pairs(const orc_admm *s);
/* Copies of the state in the layout of orc_geometry / orc_pairs:
 *   which = 0: u   (concatenated subdomain rectangles, d ascending)
 *           1: Gamma (J x m x m, natural frequency order)
 *           2: Lambda (concatenated pair rectangles, pair order)
 *           3: W_d (D x m x m, blind; the known probe repeated when nonblind)
 *           4: Delta_d (D x m x m, blind; zeros when nonblind)
 *           5: w (m x m shared probe)
 *           6: v (concatenated pair rectangles; v_{d,e} = v_{e,d})
 *           7: z of the last iteration (J x m x m)                              */
int64_t orc_admm_state_len(const orc_admm *s, int which);
void orc_admm_get(const orc_admm *s, int which, ocplx *out);
void orc_admm_set(orc_admm *s, int which, const ocplx *in);
/* Ownership mask (D entries, nonzero = owned; NULL = all): an iteration then
 * updates only the owned subdomains and reads the others' u, Lambda, W_d and
 * Delta_d as last set (halo copies of another instance's subdomains).       */
void orc_admm_set_owned(orc_admm *s, const int32_t *owned);
/* RF of the iterate entering the last iteration and RE of the last update. */
void orc_admm_metrics(const orc_admm *s, double *rf, double *re);
/* Merged image (section 4 set-up: overlaps averaged) and shared probe. */
/* Penalty change between iterations, keeping the unscaled multipliers
 * (Gamma <- eta/eta' Gamma, Lambda <- r/r' Lambda); consensus residual
 * ||u_d - u_e|| over the ordered pairs' overlaps relative to ||u||.          */
void orc_admm_set_penalties(orc_admm *s, double eta, double r);
double orc_admm_consensus(const orc_admm *s);
void orc_admm_merge(const orc_admm *s, ocplx *u_out);

#endif
