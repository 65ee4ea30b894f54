// Device helpers shared by the frame-space kernels (complex arithmetic, the
// in-register DFTs, the ST-AGM prox and fixed-order block sums).
#pragma once

#include <cuda_runtime.h>

namespace od2p {
namespace {

// Complex add / subtract as one packed FP32x2 instruction each (sm_100+):
// per component exactly a + b and a - b (b * -1 is exact, one rounding).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
#ifdef OD2P_PACKED_CMUL
// a * b as one packed multiply and one packed fused multiply-add:
// (a.x b.x, a.x b.y) + a.y (-b.y, b.x)
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return __ffma2_rn(make_float2(a.y, a.y), make_float2(-b.y, b.x), __fmul2_rn(make_float2(a.x, a.x), b));
}
// a * conj(b) = (a.x b.x, -a.x b.y) + a.y (b.y, b.x)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return __ffma2_rn(make_float2(a.y, a.y), make_float2(b.y, b.x),
                      __fmul2_rn(make_float2(a.x, a.x), make_float2(b.x, -b.y)));
}
#else
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
#endif
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

__host__ __device__ constexpr int brev(int i, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

// v * exp(-+2 pi i n / 16) for n in [0, 8) (forward: minus).  cos(pi/8), sin(pi/8)
// and sqrt(1/2) are the exact values rounded to float.
template <bool INV>
__device__ __forceinline__ float2 tw16(float2 v, int n)
{
    constexpr float C1 = 0.92387953251128674f, S1 = 0.38268343236508977f, H = 0.70710678118654752f;
    const float sg = INV ? 1.f : -1.f;
    switch (n) {
    case 0: return v;
    case 1: return cmul(v, make_float2(C1, sg * S1));
    case 2: return cscale(make_float2(v.x - sg * v.y, v.y + sg * v.x), H);
    case 3: return cmul(v, make_float2(S1, sg * C1));
    case 4: return make_float2(-sg * v.y, sg * v.x);
    case 5: return cmul(v, make_float2(-S1, sg * C1));
    case 6: return cscale(make_float2(-v.x - sg * v.y, -v.y + sg * v.x), H);
    default: return cmul(v, make_float2(-C1, sg * S1));
    }
}

// In-register R-point DFT for R a power of two (R <= 16), natural order in
// and out, unnormalised: a radix-2 network with exact twiddle constants.
template <int R, bool INV>
__device__ __forceinline__ void dft_pow2(float2 (&x)[R])
{
#pragma unroll
    for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
        for (int blk = 0; blk < R; blk += 2 * span) {
#pragma unroll
            for (int k = 0; k < span; ++k) {
                const float2 a = x[blk + k], b = x[blk + k + span];
                x[blk + k] = cadd(a, b);
                x[blk + k + span] = tw16<INV>(csub(a, b), k * (16 / (2 * span)));
            }
        }
    }
    float2 y[R];
#pragma unroll
    for (int i = 0; i < R; ++i) y[i] = x[brev(i, ilog2(R))];
#pragma unroll
    for (int i = 0; i < R; ++i) x[i] = y[i];
}

// cos and sin of d degrees for d a multiple of 18 or 30 (the angles of the 3-,
// 5-, 6-, 10- and 12-point DFTs), from their closed forms:
// cos 30 = sqrt(3)/2, cos 36 = (1 + sqrt(5))/4, cos 72 = (sqrt(5) - 1)/4.
__host__ __device__ constexpr float2 unit_deg(int d)
{
    d = ((d % 360) + 360) % 360;
    const int q = d / 90, r = d % 90;
    constexpr double R3 = 0.86602540378443864676, C36 = 0.80901699437494742410, S36 = 0.58778525229247312917,
                     C72 = 0.30901699437494742410, S72 = 0.95105651629515357212;
    double c = 1.0, s = 0.0;
    if (r == 18) c = S72, s = C72;
    else if (r == 30) c = R3, s = 0.5;
    else if (r == 36) c = C36, s = S36;
    else if (r == 54) c = S36, s = C36;
    else if (r == 60) c = 0.5, s = R3;
    else if (r == 72) c = C72, s = S72;
    // rotate by q quarter turns
    const double cq = q == 0 ? c : q == 1 ? -s : q == 2 ? -c : s;
    const double sq = q == 0 ? s : q == 1 ? c : q == 2 ? -s : -c;
    return float2{(float)cq, (float)sq};
}

// v * exp(-+2 pi i e / R) (forward: minus) for the small radices above
template <int R, bool INV>
__device__ __forceinline__ float2 twR(float2 v, int e)
{
    const float2 u = unit_deg((INV ? 360 : -360) * (e % R) / R);
    if (e % R == 0) return v;
    return cmul(v, u);
}

// Direct R-point DFT (R = 3 or 5): X_k = sum_n x_n exp(-+2 pi i n k / R).
template <int R, bool INV>
__device__ __forceinline__ void dft_direct(float2 (&x)[R])
{
    float2 y[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        float2 acc = x[0];
#pragma unroll
        for (int n = 1; n < R; ++n) acc = cadd(acc, twR<R, INV>(x[n], n * k));
        y[k] = acc;
    }
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = y[k];
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2 (&x)[R]);

// Cooley-Tukey R = A * B: X[k1 + A k2] = sum_{n2 < B} W_B^{n2 k2} W_R^{n2 k1}
// sum_{n1 < A} x[B n1 + n2] W_A^{n1 k1}.
template <int A, int B, bool INV>
__device__ __forceinline__ void dft_ct(float2 (&x)[A * B])
{
    constexpr int R = A * B;
    float2 t[B][A];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) {
        float2 v[A];
#pragma unroll
        for (int n1 = 0; n1 < A; ++n1) v[n1] = x[B * n1 + n2];
        dft<A, INV>(v);
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) t[n2][k1] = twR<R, INV>(v[k1], n2 * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
        float2 v[B];
#pragma unroll
        for (int n2 = 0; n2 < B; ++n2) v[n2] = t[n2][k1];
        dft<B, INV>(v);
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) x[k1 + A * k2] = v[k2];
    }
}

// In-register R-point DFT, natural order in and out, unnormalised:
// R in {2, 4, 8, 16} (radix-2 network), 3, 5 (direct), 6 = 2 x 3, 12 = 4 x 3.
template <int R, bool INV>
__device__ __forceinline__ void dft(float2 (&x)[R])
{
    if constexpr ((R & (R - 1)) == 0) {
        dft_pow2<R, INV>(x);
    } else if constexpr (R == 3 || R == 5) {
        dft_direct<R, INV>(x);
    } else if constexpr (R == 6) {
        dft_ct<2, 3, INV>(x);
    } else {
        static_assert(R == 12, "supported DFT lengths: 2, 3, 4, 5, 6, 8, 12, 16");
        dft_ct<4, 3, INV>(x);
    }
}

__device__ __forceinline__ float block_sum_fixed(float v, float *red)
{
    // fixed-order reduction: xor butterflies inside each warp, then warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    return t;
}

// eq. (Prox_sol) with the threshold read as |y| < (eps - (1-eps)/lam) sqrt f.
// z = y * rho / |y| with 1/|y| from the hardware reciprocal square root
// (relative error ~1e-7, far inside the FP32 parity budget); y = 0 gives (rho, 0).
__device__ __forceinline__ float2 stagm_prox(float2 y, float sf, const ProxConst &k)
{
    const float y2 = y.x * y.x + y.y * y.y;
    const float inv = rsqrtf(y2);  // +inf at y = 0, used only when y2 > 0
    const float ay = y2 > 0.f ? y2 * inv : 0.f;
    float rho;
    if (ay < k.c_thr * sf)
        rho = fmaxf(0.f, k.c_k1 * ay);
    else
        rho = (sf + k.lam * ay) * k.inv1plam;
    if (y2 > 0.f) {
        const float sc = rho * inv;
        return make_float2(y.x * sc, y.y * sc);
    }
    return make_float2(rho, 0.f);
}



}  // namespace
}  // namespace od2p
