/*
 * Forward operator A, its adjoint A^*, and the ST-AGM loss with gradients
 * (TEST INFRASTRUCTURE ONLY).
 *
 * Section 2, problem (PtychoPR): frame j is F(w o S_j u), where S_j cuts the
 * m x m window whose top-left pixel is offs[j] (integer shift, no wrap-around:
 * the image is not periodic, section 4 set-up).  A stacks all frames.
 * A^* y = sum_j S_j^T (conj(w) o F^* y_j) follows from F being unitary and S_j
 * being a 0/1 selection.  The windows are accumulated in ascending j.
 * The _ext variants take `periodic`: then S_j reads and S_j^T adds at pixel
 * ((offs[j] + a) mod H, (offs[j] + b) mod W) (the torus reading of the
 * periodic boundary in geometry.c); the plain functions are periodic = 0.
 */
#include "od2p_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* index of window pixel (r0 + r, c0 + c) in the H x W image */
static inline size_t pix(int H, int W, int periodic, int R, int C)
{
    if (periodic) {
        R %= H;
        C %= W;
        if (R < 0) R += H;
        if (C < 0) C += W;
    }
    return (size_t)R * W + C;
}

void orc_forward_ext(int H, int W, const ocplx *u, int m, const ocplx *w, int J,
                     const int32_t *offs, int periodic, ocplx *out)
{
    const int mm = m * m;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < J; ++j) {
        ocplx *x = out + (size_t)j * mm;
        const int r0 = offs[2 * j], c0 = offs[2 * j + 1];
        for (int r = 0; r < m; ++r)
            for (int c = 0; c < m; ++c)
                x[r * m + c] = w[r * m + c] * u[pix(H, W, periodic, r0 + r, c0 + c)];
        orc_fft2(x, m, 0);
    }
}

void orc_forward(int H, int W, const ocplx *u, int m, const ocplx *w, int J,
                 const int32_t *offs, ocplx *out)
{
    orc_forward_ext(H, W, u, m, w, J, offs, 0, out);
}

void orc_adjoint_ext(int H, int W, int m, const ocplx *w, int J, const int32_t *offs, int periodic,
                     const ocplx *y, ocplx *u_out)
{
    const int mm = m * m;
    ocplx *q = (ocplx *)malloc(sizeof(ocplx) * (size_t)J * mm);
    memcpy(q, y, sizeof(ocplx) * (size_t)J * mm);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < J; ++j) {
        ocplx *x = q + (size_t)j * mm;
        orc_fft2(x, m, 1);
        for (int k = 0; k < mm; ++k) x[k] *= conj(w[k]);
    }
    memset(u_out, 0, sizeof(ocplx) * (size_t)H * W);
    for (int j = 0; j < J; ++j) {
        const int r0 = offs[2 * j], c0 = offs[2 * j + 1];
        for (int r = 0; r < m; ++r)
            for (int c = 0; c < m; ++c)
                u_out[pix(H, W, periodic, r0 + r, c0 + c)] += q[(size_t)j * mm + r * m + c];
    }
    free(q);
}

void orc_adjoint(int H, int W, int m, const ocplx *w, int J, const int32_t *offs,
                 const ocplx *y, ocplx *u_out)
{
    orc_adjoint_ext(H, W, m, w, J, offs, 0, y, u_out);
}

/*
 * loss(u, w) = sum_j G_eps(F(w o S_j u); f_j)   (eqs. STAGM, obj-1)
 * grad_u = sum_j S_j^T (conj(w) o F^* grad g)      (chain rule through A)
 * grad_w = sum_j conj(S_j u) o F^* grad g           (chain rule through w)
 * with grad g from eq. (objgrad).
 */
double orc_loss_grad_ext(int H, int W, const ocplx *u, int m, const ocplx *w, int J,
                         const int32_t *offs, int periodic, const double *f, double eps, ocplx *gu, ocplx *gw)
{
    const int mm = m * m;
    ocplx *x = (ocplx *)malloc(sizeof(ocplx) * (size_t)J * mm);
    double *lj = (double *)malloc(sizeof(double) * (size_t)J);
    orc_forward_ext(H, W, u, m, w, J, offs, periodic, x);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < J; ++j) {
        double acc = 0.0;
        ocplx *xj = x + (size_t)j * mm;
        const double *fj = f + (size_t)j * mm;
        for (int k = 0; k < mm; ++k) {
            acc += orc_stagm_g(xj[k], fj[k], eps);
            xj[k] = orc_stagm_grad(xj[k], fj[k], eps);
        }
        orc_fft2(xj, m, 1);
        lj[j] = acc;
    }
    double loss = 0.0;
    for (int j = 0; j < J; ++j) loss += lj[j];
    if (gu) {
        memset(gu, 0, sizeof(ocplx) * (size_t)H * W);
        for (int j = 0; j < J; ++j) {
            const int r0 = offs[2 * j], c0 = offs[2 * j + 1];
            for (int r = 0; r < m; ++r)
                for (int c = 0; c < m; ++c)
                    gu[pix(H, W, periodic, r0 + r, c0 + c)] +=
                        conj(w[r * m + c]) * x[(size_t)j * mm + r * m + c];
        }
    }
    if (gw) {
        memset(gw, 0, sizeof(ocplx) * (size_t)mm);
        for (int j = 0; j < J; ++j) {
            const int r0 = offs[2 * j], c0 = offs[2 * j + 1];
            for (int r = 0; r < m; ++r)
                for (int c = 0; c < m; ++c)
                    gw[r * m + c] += conj(u[pix(H, W, periodic, r0 + r, c0 + c)]) *
                                     x[(size_t)j * mm + r * m + c];
        }
    }
    free(x);
    free(lj);
    return loss;
}

double orc_loss_grad(int H, int W, const ocplx *u, int m, const ocplx *w, int J,
                     const int32_t *offs, const double *f, double eps, ocplx *gu, ocplx *gw)
{
    return orc_loss_grad_ext(H, W, u, m, w, J, offs, 0, f, eps, gu, gw);
}

void orc_probe_init(int m, int J, const double *f, ocplx *w0)
{
    const int mm = m * m;
    ocplx *a = (ocplx *)malloc(sizeof(ocplx) * (size_t)mm);
    for (int k = 0; k < mm; ++k) w0[k] = 0.0;
    for (int j = 0; j < J; ++j) {
        const double *fj = f + (size_t)j * mm;
        for (int k = 0; k < mm; ++k) a[k] = sqrt(fj[k]);
        orc_fft2(a, m, 1);  /* F^* sqrt(f_j) */
        for (int k = 0; k < mm; ++k) w0[k] += a[k];
    }
    for (int k = 0; k < mm; ++k) w0[k] /= (double)J;
    free(a);
}

/* Section 4's signal-to-noise ratio SNR(u_r, u_g) = -10 log10(||u_r - u_g||^2 /
 * ||u_r||^2) dB, u_r the recovery and u_g the ground truth (the paper's naming,
 * denominator included), after removing the recovery's global phase:
 * u_r <- e^{i theta} u_r, theta = arg sum conj(u_r) u_g. */
double orc_snr(int64_t n, const ocplx *ur, const ocplx *ug)
{
    ocplx c = 0.0;
    for (int64_t k = 0; k < n; ++k) c += conj(ur[k]) * ug[k];
    const ocplx ph = cabs(c) > 0.0 ? c / cabs(c) : 1.0;
    double num = 0.0, den = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        const ocplx d = ph * ur[k] - ug[k];
        num += creal(d) * creal(d) + cimag(d) * cimag(d);
        den += creal(ur[k]) * creal(ur[k]) + cimag(ur[k]) * cimag(ur[k]);
    }
    return -10.0 * log10(num / den);
}
