/*
 * Unitary 2-D DFT for the oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Section 2 defines F as the normalized discrete Fourier transform of an
 * m x m frame.  Reading: unitary scaling 1/m (= 1/sqrt(m*m)) in both
 * directions, natural frequency order, forward kernel exp(-2 pi i k n / m).
 *
 * orc_dft2 is the definition written out (O(m^4)); orc_fft2 applies a 1-D
 * transform to every row and then every column: a textbook iterative radix-2
 * Cooley-Tukey FFT when m is a power of two, else the 1-D definition (O(m^2)
 * per line).  The tests pin each against the other and against numpy.
 */
#include "od2p_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

void orc_dft2(ocplx *x, int m, int inverse)
{
    const double sgn = inverse ? 1.0 : -1.0;
    ocplx *out = (ocplx *)malloc(sizeof(ocplx) * (size_t)m * m);
    for (int k1 = 0; k1 < m; ++k1)
        for (int k2 = 0; k2 < m; ++k2) {
            ocplx acc = 0.0;
            for (int n1 = 0; n1 < m; ++n1)
                for (int n2 = 0; n2 < m; ++n2) {
                    /* reduce the phase index mod m before scaling: exact angle */
                    long ph = ((long)k1 * n1 + (long)k2 * n2) % m;
                    double a = sgn * 2.0 * ORC_PI * (double)ph / (double)m;
                    acc += x[n1 * m + n2] * (cos(a) + I * sin(a));
                }
            out[k1 * m + k2] = acc / (double)m;
        }
    memcpy(x, out, sizeof(ocplx) * (size_t)m * m);
    free(out);
}

/* In-place radix-2 FFT of n points spaced `stride` apart (unnormalised). */
static void fft1(ocplx *x, int n, int stride, int inverse)
{
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            ocplx t = x[i * stride];
            x[i * stride] = x[j * stride];
            x[j * stride] = t;
        }
    }
    const double sgn = inverse ? 1.0 : -1.0;
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1;
        for (int k = 0; k < half; ++k) {
            double a = sgn * 2.0 * ORC_PI * (double)k / (double)len;
            ocplx wk = cos(a) + I * sin(a);
            for (int i = 0; i < n; i += len) {
                ocplx p = x[(i + k) * stride];
                ocplx q = x[(i + k + half) * stride] * wk;
                x[(i + k) * stride] = p + q;
                x[(i + k + half) * stride] = p - q;
            }
        }
    }
}

/* The 1-D DFT of n points spaced `stride` apart, by its definition (unnormalised). */
static void dft1(ocplx *x, int n, int stride, int inverse)
{
    const double sgn = inverse ? 1.0 : -1.0;
    ocplx *out = (ocplx *)malloc(sizeof(ocplx) * (size_t)n);
    for (int k = 0; k < n; ++k) {
        ocplx acc = 0.0;
        for (int t = 0; t < n; ++t) {
            const long ph = ((long)k * t) % n;
            const double a = sgn * 2.0 * ORC_PI * (double)ph / (double)n;
            acc += x[t * stride] * (cos(a) + I * sin(a));
        }
        out[k] = acc;
    }
    for (int k = 0; k < n; ++k) x[k * stride] = out[k];
    free(out);
}

void orc_fft2(ocplx *x, int m, int inverse)
{
    const int pow2 = m > 0 && (m & (m - 1)) == 0;
    for (int r = 0; r < m; ++r) {
        if (pow2)
            fft1(x + (size_t)r * m, m, 1, inverse);
        else
            dft1(x + (size_t)r * m, m, 1, inverse);
    }
    for (int c = 0; c < m; ++c) {
        if (pow2)
            fft1(x + c, m, m, inverse);
        else
            dft1(x + c, m, m, inverse);
    }
    const double s = 1.0 / (double)m;
    for (int i = 0; i < m * m; ++i) x[i] *= s;
}
