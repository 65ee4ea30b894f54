/*
 * Smooth-truncated amplitude-Gaussian metric (ST-AGM), section 2.2
 * (TEST INFRASTRUCTURE ONLY).
 *
 * g_eps(x; b), eq. (obj-1):
 *   (1-eps)/2 * (b - |x|^2/eps)   if |x| < eps*sqrt(b)      (region K1)
 *   1/2 * (|x| - sqrt(b))^2       otherwise                 (region K2)
 *
 * Gradient, eq. (objgrad) (convention d/dRe + i d/dIm):
 *   (1 - 1/eps) x in K1,  (1 - sqrt(b)/|x|) x in K2.
 *
 * Proximal map, eq. (Prox_sol).  The threshold is garbled in the paper; the
 * reading used is |y| < (eps - (1-eps)/lam) * sqrt(f), which is where the K2
 * stationary point (sqrt(f) + lam|y|)/(1+lam) stops being admissible
 * (minimise g(rho e^{i arg y}) + lam/2 (rho - |y|)^2 over rho >= 0).  The K1
 * branch lam|y| / (lam - (1-eps)/eps) is reached only when
 * lam > (1-eps)/eps.  sign(0) is read as 1 (any phase is optimal there).
 */
#include "od2p_oracle.h"

#include <math.h>

double orc_stagm_g(ocplx x, double b, double eps)
{
    double ax = cabs(x), sb = sqrt(b);
    if (ax < eps * sb) return 0.5 * (1.0 - eps) * (b - ax * ax / eps);
    return 0.5 * (ax - sb) * (ax - sb);
}

ocplx orc_stagm_grad(ocplx x, double b, double eps)
{
    double ax = cabs(x), sb = sqrt(b);
    if (ax < eps * sb) return (1.0 - 1.0 / eps) * x;
    if (ax == 0.0) return 0.0; /* b == 0 and x == 0: g = |x|^2/2, gradient 0 */
    return (1.0 - sb / ax) * x;
}

ocplx orc_stagm_prox(ocplx y, double f, double eps, double lam)
{
    double ay = cabs(y), sf = sqrt(f);
    ocplx sgn = ay > 0.0 ? y / ay : 1.0;
    double thr = (eps - (1.0 - eps) / lam) * sf;
    double rho;
    if (ay < thr) {
        rho = lam * ay / (lam - (1.0 - eps) / eps);
        if (rho < 0.0) rho = 0.0;
    } else {
        rho = (sf + lam * ay) / (1.0 + lam);
    }
    return sgn * rho;
}

void orc_stagm_g_arr(const ocplx *x, const double *b, int64_t n, double eps, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_stagm_g(x[i], b[i], eps);
}

void orc_stagm_grad_arr(const ocplx *x, const double *b, int64_t n, double eps, ocplx *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_stagm_grad(x[i], b[i], eps);
}

void orc_stagm_prox_arr(const ocplx *y, const double *f, int64_t n, double eps, double lam,
                        ocplx *z)
{
    for (int64_t i = 0; i < n; ++i) z[i] = orc_stagm_prox(y[i], f[i], eps, lam);
}
