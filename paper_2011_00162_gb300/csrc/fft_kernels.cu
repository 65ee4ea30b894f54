// Frame-space kernels of the OD2P library for sm_103a: the fused frame update
// (exit wave -> unitary 2-D FFT -> ST-AGM prox + Gamma update -> inverse FFT),
// the forward operator, the frame inverse-FFT of the adjoint, the loss frames,
// and the blind probe average.  No tensor cores: the work is FFT butterflies
// and elementwise arithmetic, bound by HBM and shared memory.
//
// 2-D FFT scheme.  An m x m frame lives in shared memory with an odd row pitch
// P = m + 1.  The length-m transform is split m = R1 * R2 (Cooley-Tukey,
// decimation in frequency):
//   stage 1: for n1 < R2, R1-point DFT over x[n1 + R2 t], times exp(-2 pi i n1 s / m),
//            stored at n1 + R2 s;
//   stage 2: for s < R1, R2-point DFT over the contiguous block [R2 s, R2 s + R2);
// so position p = R2 s + s' holds frequency k = s + R1 s' (digit-reversed).
// The 2-D transform runs stage 1 and 2 along columns (lanes on columns:
// coalesced global loads, conflict-free shared rows) and then along rows
// (lanes on rows: the odd pitch makes them conflict-free).  The inverse is the
// exact adjoint, stages in reverse order, so natural order comes back without
// any bit-reversal pass.  Frequency-space arrays private to the plan (Gamma,
// sqrt f) are stored in the order the row stage holds them: element
// (position row pr, position column pc) at pc * m + pr, which makes the
// prox's loads and stores coalesced.  Each R-point DFT runs in registers as a
// radix-2 network with exact twiddle constants.
#include "od2p_internal.h"
#include "fft_device.cuh"

#include <cmath>
#include <mutex>
#include <string>

namespace od2p {
namespace {

template <int M> struct Radix;
// R1 x R2 split, frames per block, threads per block, and the resident blocks
// per SM the register budget is sized for (shared memory allows the same).
template <> struct Radix<16> { static constexpr int R1 = 4, R2 = 4, FPB = 8, NT = 256, MINB = 6; };
template <> struct Radix<32> { static constexpr int R1 = 8, R2 = 4, FPB = 4, NT = 256, MINB = 6; };
#ifndef OD2P_NT64
#define OD2P_NT64 256
#endif
#ifndef OD2P_MINB64
#define OD2P_MINB64 6
#endif
template <> struct Radix<64> { static constexpr int R1 = 8, R2 = 8, FPB = 1, NT = OD2P_NT64, MINB = OD2P_MINB64; };
template <> struct Radix<128> { static constexpr int R1 = 16, R2 = 8, FPB = 1, NT = 1024, MINB = 1; };
// probe sides that are not powers of two: mixed-radix splits (stage 2 uses the
// 6-, 5- and 12-point DFTs)
template <> struct Radix<48> { static constexpr int R1 = 8, R2 = 6, FPB = 2, NT = 384, MINB = 1; };
template <> struct Radix<80> { static constexpr int R1 = 16, R2 = 5, FPB = 1, NT = 448, MINB = 1; };
template <> struct Radix<96> { static constexpr int R1 = 8, R2 = 12, FPB = 1, NT = 384, MINB = 1; };

// Ask the TMA unit to stage [p, p + bytes) into L2 (bytes a multiple of 16,
// p 16-byte aligned); issued early so the data is near when it is needed.
__device__ __forceinline__ void bulk_prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int M> constexpr size_t smem_bytes()
{
    return sizeof(float2) * (M + (size_t)Radix<M>::FPB * M * (M + 1)) +
           sizeof(float) * (Radix<M>::NT / 32);
}

// position <-> frequency along one axis
template <int M> __device__ __forceinline__ int pos_of(int k)
{
    return Radix<M>::R2 * (k % Radix<M>::R1) + k / Radix<M>::R1;
}

// ---------------------------------------------------------------- shared stages
// Column-direction stage 2 (forward or inverse) over all FPB frames.
template <int M, bool INV, int FPB = Radix<M>::FPB, int NT = Radix<M>::NT>
__device__ __forceinline__ void col_stage2(float2 *buf)
{
    constexpr int R1 = Radix<M>::R1, R2 = Radix<M>::R2;
    constexpr int P = M + 1;
    for (int task = threadIdx.x; task < FPB * M * R1; task += NT) {
        const int c = task % M, rest = task / M, s = rest % R1, f = rest / R1;
        float2 *fb = buf + f * M * P;
        float2 x[R2];
#pragma unroll
        for (int t = 0; t < R2; ++t) x[t] = fb[(R2 * s + t) * P + c];
        dft<R2, INV>(x);
#pragma unroll
        for (int t = 0; t < R2; ++t) fb[(R2 * s + t) * P + c] = x[t];
    }
}

// Row-direction stage 1, forward (DFT then twiddle) or inverse (twiddle then DFT).
template <int M, bool INV, int FPB = Radix<M>::FPB, int NT = Radix<M>::NT>
__device__ __forceinline__ void row_stage1(float2 *buf, const float2 *tw)
{
    constexpr int R1 = Radix<M>::R1, R2 = Radix<M>::R2;
    constexpr int P = M + 1;
    for (int task = threadIdx.x; task < FPB * M * R2; task += NT) {
        const int r = task % M, rest = task / M, n1 = rest % R2, f = rest / R2;
        float2 *fb = buf + f * M * P + r * P;
        float2 x[R1];
        if (!INV) {
#pragma unroll
            for (int t = 0; t < R1; ++t) x[t] = fb[n1 + R2 * t];
            dft<R1, false>(x);
#pragma unroll
            for (int s = 0; s < R1; ++s) fb[n1 + R2 * s] = cmul(x[s], tw[n1 * s]);
        } else {
#pragma unroll
            for (int s = 0; s < R1; ++s) x[s] = cmulc(fb[n1 + R2 * s], tw[n1 * s]);
            dft<R1, true>(x);
#pragma unroll
            for (int t = 0; t < R1; ++t) fb[n1 + R2 * t] = x[t];
        }
    }
}

// Column-direction stage 1 reading / writing shared memory.
template <int M, bool INV, int FPB = Radix<M>::FPB, int NT = Radix<M>::NT>
__device__ __forceinline__ void col_stage1(float2 *buf, const float2 *tw)
{
    constexpr int R1 = Radix<M>::R1, R2 = Radix<M>::R2;
    constexpr int P = M + 1;
    for (int task = threadIdx.x; task < FPB * M * R2; task += NT) {
        const int c = task % M, rest = task / M, n1 = rest % R2, f = rest / R2;
        float2 *fb = buf + f * M * P;
        float2 x[R1];
        if (!INV) {
#pragma unroll
            for (int t = 0; t < R1; ++t) x[t] = fb[(n1 + R2 * t) * P + c];
            dft<R1, false>(x);
#pragma unroll
            for (int s = 0; s < R1; ++s) fb[(n1 + R2 * s) * P + c] = cmul(x[s], tw[n1 * s]);
        } else {
#pragma unroll
            for (int s = 0; s < R1; ++s) x[s] = cmulc(fb[(n1 + R2 * s) * P + c], tw[n1 * s]);
            dft<R1, true>(x);
#pragma unroll
            for (int t = 0; t < R1; ++t) fb[(n1 + R2 * t) * P + c] = x[t];
        }
    }
}

// Row-direction stage 2 in shared memory (forward or inverse).
template <int M, bool INV, int FPB = Radix<M>::FPB, int NT = Radix<M>::NT>
__device__ __forceinline__ void row_stage2(float2 *buf)
{
    constexpr int R1 = Radix<M>::R1, R2 = Radix<M>::R2;
    constexpr int P = M + 1;
    for (int task = threadIdx.x; task < FPB * M * R1; task += NT) {
        const int r = task % M, rest = task / M, s = rest % R1, f = rest / R1;
        float2 *fb = buf + f * M * P + r * P;
        float2 x[R2];
#pragma unroll
        for (int t = 0; t < R2; ++t) x[t] = fb[R2 * s + t];
        dft<R2, INV>(x);
#pragma unroll
        for (int t = 0; t < R2; ++t) fb[R2 * s + t] = x[t];
    }
}

// Column stage 1 whose input is the exit wave w o S_j u read from global memory.
template <int M, int FPB = Radix<M>::FPB, int NT = Radix<M>::NT>
__device__ __forceinline__ void col_stage1_load(float2 *buf, const float2 *tw, int j0, int J,
                                                const float2 *w_shared, const float2 *Wd,
                                                const int32_t *frame_sub, const float2 *u,
                                                const int32_t *frame_base, const int32_t *frame_pitch)
{
    constexpr int R1 = Radix<M>::R1, R2 = Radix<M>::R2;
    constexpr int P = M + 1;
    for (int task = threadIdx.x; task < FPB * M * R2; task += NT) {
        const int c = task % M, rest = task / M, n1 = rest % R2, f = rest / R2, j = j0 + f;
        if (j >= J) continue;
        const float2 *w = Wd ? Wd + (size_t)frame_sub[j] * M * M : w_shared;
        const float2 *uj = u + frame_base[j];
        const int pitch = frame_pitch[j];
        float2 x[R1];
#pragma unroll
        for (int t = 0; t < R1; ++t) {
            const int row = n1 + R2 * t;
            x[t] = cmul(__ldg(w + row * M + c), __ldg(uj + (size_t)row * pitch + c));
        }
        dft<R1, false>(x);
        float2 *fb = buf + f * M * P;
#pragma unroll
        for (int s = 0; s < R1; ++s) fb[(n1 + R2 * s) * P + c] = cmul(x[s], tw[n1 * s]);
    }
}

// Column stage 1^H writing natural-order frames to global memory, scaled by
// `scale` and, when wconj is given, multiplied by conj(wconj).
template <int M, int FPB = Radix<M>::FPB, int NT = Radix<M>::NT>
__device__ __forceinline__ void col_stage1_store(float2 *buf, const float2 *tw, int j0, int J,
                                                 float2 *out, float scale, const float2 *wconj)
{
    constexpr int R1 = Radix<M>::R1, R2 = Radix<M>::R2;
    constexpr int P = M + 1;
    for (int task = threadIdx.x; task < FPB * M * R2; task += NT) {
        const int c = task % M, rest = task / M, n1 = rest % R2, f = rest / R2, j = j0 + f;
        if (j >= J) continue;
        float2 *fb = buf + f * M * P;
        float2 x[R1];
#pragma unroll
        for (int s = 0; s < R1; ++s) x[s] = cmulc(fb[(n1 + R2 * s) * P + c], tw[n1 * s]);
        dft<R1, true>(x);
        float2 *o = out + (size_t)j * M * M;
#pragma unroll
        for (int t = 0; t < R1; ++t) {
            const int row = n1 + R2 * t;
            float2 v = cscale(x[t], scale);
            if (wconj) v = cmulc(v, __ldg(wconj + row * M + c));
            o[row * M + c] = v;
        }
    }
}

// Slot ranks of a thread's column tasks, loaded at the start of a frame group
// and used at its end (the loads complete while the FFT runs).  Ranks are
// stored in task order: task (n1, c) of frame j holds the R1 ranks of rows
// n1 + R2 t, t < R1, at rank[j m^2 + (n1 m + c) R1 + t].
template <int M, int FPB, int NT>
struct SlotRanks {
    static constexpr int R1 = Radix<M>::R1, R2 = Radix<M>::R2;
    static constexpr int TASKS = FPB * M * R2, TPT = (TASKS + NT - 1) / NT, WPT = R1 / 4;
    static_assert(R1 % 4 == 0, "ranks are loaded four at a time");
    uint32_t w[TPT][WPT];

    __device__ __forceinline__ void load(const uint8_t *rank, int j0, int J)
    {
#pragma unroll
        for (int i = 0; i < TPT; ++i) {
            const int task = threadIdx.x + i * NT;
            const int c = task % M, rest = task / M, n1 = rest % R2, f = rest / R2, j = j0 + f;
            const bool ok = task < TASKS && j < J;
            const uint8_t *src = rank + (size_t)(ok ? j : 0) * M * M + ((size_t)n1 * M + c) * R1;
            if constexpr (WPT == 1) {
                w[i][0] = ok ? __ldg(reinterpret_cast<const uint32_t *>(src)) : 0u;
            } else if constexpr (WPT == 2) {
                const uint2 v = ok ? __ldg(reinterpret_cast<const uint2 *>(src)) : make_uint2(0u, 0u);
                w[i][0] = v.x;
                w[i][1] = v.y;
            } else {
                static_assert(WPT == 4, "R1 is 4, 8 or 16");
                const uint4 v = ok ? __ldg(reinterpret_cast<const uint4 *>(src)) : make_uint4(0u, 0u, 0u, 0u);
                w[i][0] = v.x;
                w[i][1] = v.y;
                w[i][2] = v.z;
                w[i][3] = v.w;
            }
        }
    }
    __device__ __forceinline__ unsigned get(int i, int t) const { return (w[i][t / 4] >> (8 * (t % 4))) & 0xffu; }
};

// Column stage 1^H writing conj(w) o (natural-order frame) into the gather
// slots: frame j's pixel (row, c) goes to slot[rank * stride + base_j + row *
// pitch_j + c], the ranks taken from the preloaded registers.
template <int M, int FPB, int NT>
__device__ __forceinline__ void col_stage1_store_slots(float2 *buf, const float2 *tw, int j0, int J,
                                                       float2 *slot, const SlotRanks<M, FPB, NT> &rk, int stride,
                                                       const int32_t *frame_base, const int32_t *frame_pitch,
                                                       float scale, const float2 *w)
{
    constexpr int R1 = Radix<M>::R1, R2 = Radix<M>::R2, P = M + 1;
    constexpr int TASKS = FPB * M * R2, TPT = SlotRanks<M, FPB, NT>::TPT;
#pragma unroll
    for (int i = 0; i < TPT; ++i) {
        const int task = threadIdx.x + i * NT;
        if (task >= TASKS) break;
        const int c = task % M, rest = task / M, n1 = rest % R2, f = rest / R2, j = j0 + f;
        if (j >= J) continue;
        float2 *fb = buf + f * M * P;
        float2 x[R1];
#pragma unroll
        for (int s = 0; s < R1; ++s) x[s] = cmulc(fb[(n1 + R2 * s) * P + c], tw[n1 * s]);
        dft<R1, true>(x);
        const unsigned base = (unsigned)(frame_base[j] + c), pitch = (unsigned)frame_pitch[j];
#pragma unroll
        for (int t = 0; t < R1; ++t) {
            const int row = n1 + R2 * t;
            const float2 v = cmulc(cscale(x[t], scale), __ldg(w + row * M + c));
            // 32-bit index: the plan checks slot_k * u_len < 2^32
            slot[rk.get(i, t) * (unsigned)stride + base + (unsigned)row * pitch] = v;
        }
    }
}

// ---------------------------------------------------------------- K1: fused frame update

// Launch shapes of the persistent frame update: frames per group, threads, and
// whether Gamma is staged in shared memory (m = 128 only stages sqrt f: the
// frame buffer already takes 132 KB).  Two shapes (variant 0 / 1) are compiled
// per probe side; the autotuner picks one per plan.  Variant 1 trades the Gamma
// staging (Gamma then comes from L2 after a bulk prefetch) for more resident
// blocks at m = 32 and 64.  MINB: resident blocks per SM the register budget
// is sized for (shared memory allows at least as many).
template <int M, int V> struct K1Cfg;
template <> struct K1Cfg<16, 0> { static constexpr int FPB = 8, NT = 256, STAGE_G = 1, MINB = 4; };
template <> struct K1Cfg<16, 1> { static constexpr int FPB = 4, NT = 128, STAGE_G = 1, MINB = 8; };
template <> struct K1Cfg<32, 0> { static constexpr int FPB = 4, NT = 256, STAGE_G = 1, MINB = 2; };
template <> struct K1Cfg<32, 1> { static constexpr int FPB = 2, NT = 128, STAGE_G = 0, MINB = 8; };
template <> struct K1Cfg<64, 0> { static constexpr int FPB = 1, NT = 512, STAGE_G = 1, MINB = 2; };
template <> struct K1Cfg<64, 1> { static constexpr int FPB = 1, NT = 512, STAGE_G = 0, MINB = 3; };
template <> struct K1Cfg<128, 0> { static constexpr int FPB = 1, NT = 1024, STAGE_G = 0, MINB = 1; };
template <> struct K1Cfg<128, 1> { static constexpr int FPB = 1, NT = 512, STAGE_G = 0, MINB = 1; };
template <> struct K1Cfg<48, 0> { static constexpr int FPB = 2, NT = 384, STAGE_G = 1, MINB = 2; };
template <> struct K1Cfg<48, 1> { static constexpr int FPB = 1, NT = 384, STAGE_G = 0, MINB = 3; };
template <> struct K1Cfg<80, 0> { static constexpr int FPB = 1, NT = 448, STAGE_G = 0, MINB = 2; };
template <> struct K1Cfg<80, 1> { static constexpr int FPB = 1, NT = 640, STAGE_G = 0, MINB = 1; };
template <> struct K1Cfg<96, 0> { static constexpr int FPB = 1, NT = 384, STAGE_G = 0, MINB = 2; };
template <> struct K1Cfg<96, 1> { static constexpr int FPB = 1, NT = 768, STAGE_G = 0, MINB = 1; };

template <int M, int V> constexpr size_t k1_smem_bytes()
{
    constexpr size_t FPB = K1Cfg<M, V>::FPB, MM = (size_t)M * M;
    return 128 + (K1Cfg<M, V>::STAGE_G ? sizeof(float2) * FPB * MM : 0) + sizeof(float) * FPB * MM +
           sizeof(float2) * (M + FPB * M * (M + 1)) + sizeof(float) * (K1Cfg<M, V>::NT / 32);
}

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// TMA bulk copy global -> shared, completing `bytes` on the mbarrier
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Every wait is bounded: after 2^22 polls (seconds) it reports failure.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity)
{
    for (int i = 0; i < (1 << 22); ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Persistent and table-driven: work item i (block b takes b, b + grid, ...)
// is frame group items[i].y of the plan whose arguments are tab[2 items[i].x
// + parity] (one plan: items = null and item i is group i of tab[parity]).
// While a group's forward FFT runs, the TMA unit brings its Gamma and sqrt f
// slices into shared memory (issued when the previous group's prox finished
// with the staging buffers), and the next group's exit-wave windows are
// prefetched into L2.  Each group's RF partial goes to rf_part[group].
template <int M, int V, bool BATCHED>
__global__ void __launch_bounds__(K1Cfg<M, V>::NT, K1Cfg<M, V>::MINB)
    frame_update_kernel(const FrameArgs single, const FrameArgs *__restrict__ tab, const int2 *__restrict__ items,
                        int n_items, int parity)
{
    constexpr int R1 = Radix<M>::R1, R2 = Radix<M>::R2, FPB = K1Cfg<M, V>::FPB, NT = K1Cfg<M, V>::NT;
    constexpr int P = M + 1, MM = M * M;
    constexpr bool SG = K1Cfg<M, V>::STAGE_G != 0;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ FrameArgs sa_batch;  // batches: arguments of the current item's plan
    const FrameArgs &sa = BATCHED ? sa_batch : single;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    float2 *stg_g = reinterpret_cast<float2 *>(smem + 128);
    float *stg_f = reinterpret_cast<float *>(smem + 128 + (SG ? sizeof(float2) * FPB * MM : 0));
    float2 *tw = reinterpret_cast<float2 *>(stg_f + FPB * MM);
    float2 *buf = tw + M;
    float *red = reinterpret_cast<float *>(buf + FPB * M * P);

    auto item = [&](int i) { return BATCHED ? items[i] : make_int2(0, i); };
    auto issue = [&](int i) {  // one thread: stage item i's Gamma / sqrt f
        const int2 it = item(i);
        const FrameArgs &ga = BATCHED ? tab[2 * it.x + parity] : single;
        const int j0 = it.y * FPB, nf = min(FPB, ga.J - j0);
        const unsigned fbytes = (unsigned)(nf * MM * sizeof(float));
        const unsigned gbytes = SG ? (unsigned)(nf * MM * sizeof(float2)) : 0u;
        mbar_expect_tx(bar, fbytes + gbytes);
        if (SG) bulk_g2s(stg_g, ga.gamma + (size_t)j0 * MM, gbytes, bar);
        bulk_g2s(stg_f, ga.sqrtf_ + (size_t)j0 * MM, fbytes, bar);
        // the next group's slot ranks, loaded at the start of that group
        if (ga.slot) bulk_prefetch_l2(ga.rank + (size_t)j0 * MM, (unsigned)(nf * MM));
    };
    auto prefetch_windows = [&](int i) {  // all threads: item i's exit-wave windows into L2
        constexpr int LINES = (M * 8 + 127) / 128 + 1;
        const int2 it = item(i);
        const FrameArgs &ga = BATCHED ? tab[2 * it.x + parity] : single;
        const int j0 = it.y * FPB;
        for (int k = threadIdx.x; k < FPB * M * LINES; k += NT) {
            const int f = k / (M * LINES), row = (k / LINES) % M, l = k % LINES, j = j0 + f;
            if (j >= ga.J) continue;
            const char *rp = reinterpret_cast<const char *>(ga.u + ga.frame_base[j] + (size_t)row * ga.frame_pitch[j]);
            prefetch_l2(rp + min(l * 128, M * 8 - 8));
        }
    };

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    for (int k = threadIdx.x; k < M; k += NT) tw[k] = (BATCHED ? tab[parity] : single).tw[k];
    __syncthreads();
    int i = blockIdx.x;
    if (threadIdx.x == 0 && i < n_items) issue(i);
    unsigned phase = 0;
    int plan_now = -1;
    const float inv_m = 1.f / (float)M;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (; i < n_items; i += gridDim.x) {
        const int2 it = item(i);
        if (BATCHED && it.x != plan_now) {  // uniform: every thread sees the same item
            __syncthreads();
            if (threadIdx.x == 0) sa_batch = tab[2 * it.x + parity];
            __syncthreads();
            plan_now = it.x;
        }
        const int j0 = it.y * FPB;
        if (i + (int)gridDim.x < n_items) prefetch_windows(i + gridDim.x);
        if (!SG && threadIdx.x == 0) {
            const int nf = min(FPB, sa.J - j0);
            const char *gp = reinterpret_cast<const char *>(sa.gamma + (size_t)j0 * MM);
            for (unsigned off = 0; off < (unsigned)(nf * MM * sizeof(float2)); off += 16384u)
                bulk_prefetch_l2(gp + off, min(16384u, (unsigned)(nf * MM * sizeof(float2)) - off));
        }
        // Step 1: psi = w o S_j u_d^n, then F psi (three of the four forward stages)
        col_stage1_load<M, FPB, NT>(buf, tw, j0, sa.J, sa.w, sa.Wd, sa.frame_sub, sa.u, sa.frame_base, sa.frame_pitch);
        SlotRanks<M, FPB, NT> ranks;
        if (sa.slot) ranks.load(sa.rank, j0, sa.J);
        __syncthreads();
        col_stage2<M, false, FPB, NT>(buf);
        __syncthreads();
        row_stage1<M, false, FPB, NT>(buf, tw);
        const bool ok = mbar_wait_bounded(bar, phase);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) *sa.err = 1;
            return;
        }
        phase ^= 1u;
        // last forward stage, prox and Gamma update, first inverse stage -- in registers
        float rf = 0.f;
        for (int task = threadIdx.x; task < FPB * M * R1; task += NT) {
            const int r = task % M, rest = task / M, s = rest % R1, f = rest / R1, j = j0 + f;
            if (j >= sa.J) continue;
            float2 *fb = buf + f * M * P + r * P;
            float2 x[R2];
#pragma unroll
            for (int t = 0; t < R2; ++t) x[t] = fb[R2 * s + t];
            const int lbase = f * MM + r;
            // Gamma from global memory (not staged): all loads before the stores
            // below, which the compiler may not move them past
            float2 gmv[SG ? 1 : R2];
            if (!SG) {
#pragma unroll
                for (int t = 0; t < R2; ++t) gmv[SG ? 0 : t] = sa.gamma[(size_t)j0 * MM + lbase + (R2 * s + t) * M];
            }
            dft<R2, false>(x);
#pragma unroll
            for (int t = 0; t < R2; ++t) {
                const int li = lbase + (R2 * s + t) * M;
                const size_t gi = (size_t)j0 * MM + li;
                const float2 ax = cscale(x[t], inv_m);   // (A_d u_d^n)_k
                const float sf = stg_f[li];
                const float2 gm = SG ? stg_g[li] : gmv[SG ? 0 : t];
                const float a2 = ax.x * ax.x + ax.y * ax.y;
                rf += fabsf((a2 > 0.f ? a2 * rsqrtf(a2) : 0.f) - sf);  // | |A_d u_d| - sqrt f |
                const float2 y = cadd(gm, ax);            // Gamma^n + A_d u_d^n
                const float2 z = stagm_prox(y, sf, sa.pc); // eq. updateZ
                const float2 gn = csub(y, z);             // eq. updateM-1-multi
                sa.gamma[gi] = gn;
                x[t] = csub(z, gn);                       // z^{n+1} - Gamma^{n+1}
            }
            dft<R2, true>(x);
#pragma unroll
            for (int t = 0; t < R2; ++t) fb[R2 * s + t] = x[t];
        }
        __syncthreads();  // staging buffers are free: start the next item's copies
        if (threadIdx.x == 0 && i + (int)gridDim.x < n_items) {
            fence_proxy_async_smem();
            issue(i + gridDim.x);
        }
        row_stage1<M, true, FPB, NT>(buf, tw);
        __syncthreads();
        col_stage2<M, true, FPB, NT>(buf);
        __syncthreads();
        if (sa.slot) {
            // nonblind: q_j = conj(w) o F^*(z - Gamma) (the A_d^* summand), stored in
            // the gather slot of each pixel
            col_stage1_store_slots<M, FPB, NT>(buf, tw, j0, sa.J, sa.slot, ranks, sa.slot_stride, sa.frame_base,
                                               sa.frame_pitch, inv_m, sa.w);
        } else {
            // blind: unweighted; the subdomain update weights with W_d^{n+1}
            col_stage1_store<M, FPB, NT>(buf, tw, j0, sa.J, sa.q, inv_m, nullptr);
        }
        // this group's RF partial, one per warp (fixed xor tree inside the warp)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rf += __shfl_xor_sync(0xffffffffu, rf, o);
        if (lane == 0) sa.rf_part[it.y * (NT / 32) + warp] = rf;
        __syncthreads();
    }
    (void)red;
}

// ---------------------------------------------------------------- K1, m = 64 as 16 x 4 by 4 x 16
// The same frame update with the 64-point transforms of both axes split as
// 64 = 16 x 4 (rows r = r1 + 16 r2, columns c = c1 + 16 c2) so that the two
// radix-4 stages of the two axes run together in one thread (a 4 x 4 block of
// the frame) and each radix-16 stage of an axis in another: two shared-memory
// exchanges per direction instead of three.  One frame per 256-thread block.
//  pass 1  thread (r1, c1): exit wave at (r1 + 16 r2, c1 + 16 c2), 4-point DFTs
//          over r2 then c2 with the twiddles w64^(r1 k1), w64^(c1 l1); stored at
//          row 16 k1 + r1, column 16 l1 + c1
//  pass 2  thread (column, k1): 16-point DFT over r1 -> k2; row frequency
//          k = k1 + 4 k2 stored at row 16 k1 + k2
//  pass 3  thread (k, l1): 16-point DFT over c1 -> l2, column frequency
//          l = l1 + 4 l2; prox and Gamma update at the storage position of
//          (k, l) shared with the 8 x 8 kernel; inverse 16-point DFT
//  passes 4, 5: the adjoints of 2 and 1, then the conj(w)-weighted residual
//          to the gather slots (or q in natural order for list-gather plans).
// Different rounding from the 8 x 8 split; selected per plan with
// ptycho_plan_set_fft.
template <int SG> struct F4Cfg { static constexpr int NT = 256, MINB = SG ? 2 : 3; };

template <int SG> constexpr size_t f4_smem_bytes()
{
    return 128 + (SG ? sizeof(float2) * 4096 : 0) + sizeof(float) * 4096 + sizeof(float2) * (64 + 64 * 65) +
           sizeof(float) * 8;
}

__device__ __forceinline__ int pos64(int f) { return 8 * (f & 7) + (f >> 3); }

// BATCHED: the work items are (plan, frame) pairs of several plans with m = 64,
// each plan's arguments read from tab[2 plan + parity] (the batches' form of
// the 16 x 4 split); otherwise item i is frame i of `single`.
template <int SG, bool BATCHED>
__global__ void __launch_bounds__(256, F4Cfg<SG>::MINB)
    frame_update_f4_kernel(const FrameArgs single, const FrameArgs *__restrict__ tab,
                           const int2 *__restrict__ items, int n_items, int parity)
{
    constexpr int M = 64, P = 65, MM = 4096, NT = 256;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ FrameArgs sa_batch;  // batches: arguments of the current item's plan
    const FrameArgs &sa = BATCHED ? sa_batch : single;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    float2 *stg_g = reinterpret_cast<float2 *>(smem + 128);
    float *stg_f = reinterpret_cast<float *>(smem + 128 + (SG ? sizeof(float2) * MM : 0));
    float2 *tw = reinterpret_cast<float2 *>(stg_f + MM);
    float2 *buf = tw + M;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

    auto item = [&](int i) { return BATCHED ? items[i] : make_int2(0, i); };
    auto args = [&](int2 it) -> const FrameArgs & { return BATCHED ? tab[2 * it.x + parity] : single; };
    auto issue = [&](int i) {  // one thread: stage item i's Gamma / sqrt f
        const int2 it = item(i);
        const FrameArgs &ga = args(it);
        const int j = it.y;
        const unsigned fbytes = (unsigned)(MM * sizeof(float));
        const unsigned gbytes = SG ? (unsigned)(MM * sizeof(float2)) : 0u;
        mbar_expect_tx(bar, fbytes + gbytes);
        if (SG) bulk_g2s(stg_g, ga.gamma + (size_t)j * MM, gbytes, bar);
        bulk_g2s(stg_f, ga.sqrtf_ + (size_t)j * MM, fbytes, bar);
        if (ga.slot) bulk_prefetch_l2(ga.rank + (size_t)j * MM, (unsigned)MM);
    };
    auto prefetch_window = [&](int i) {  // all threads: item i's exit-wave window into L2
        constexpr int LINES = (M * 8 + 127) / 128 + 1;
        const int2 it = item(i);
        const FrameArgs &ga = args(it);
        for (int k = t; k < M * LINES; k += NT) {
            const int row = k / LINES, l = k % LINES;
            const char *rp =
                reinterpret_cast<const char *>(ga.u + ga.frame_base[it.y] + (size_t)row * ga.frame_pitch[it.y]);
            prefetch_l2(rp + min(l * 128, M * 8 - 8));
        }
    };

    if (t == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    for (int k = t; k < M; k += NT) tw[k] = (BATCHED ? tab[parity] : single).tw[k];
    __syncthreads();
    int i = blockIdx.x;
    if (t == 0 && i < n_items) issue(i);
    unsigned phase = 0;
    int plan_now = -1;
    const float inv_m = 1.f / (float)M;
    for (; i < n_items; i += gridDim.x) {
        const int2 it = item(i);
        if (BATCHED && it.x != plan_now) {  // uniform: every thread sees the same item
            __syncthreads();
            if (t == 0) sa_batch = tab[2 * it.x + parity];
            __syncthreads();
            plan_now = it.x;
        }
        const int j = it.y;
        if (i + (int)gridDim.x < n_items) prefetch_window(i + gridDim.x);
        if (!SG && t == 0)
            for (unsigned off = 0; off < (unsigned)(MM * sizeof(float2)); off += 16384u)
                bulk_prefetch_l2(reinterpret_cast<const char *>(sa.gamma + (size_t)j * MM) + off, 16384u);
        // ---- pass 1: exit wave, 4 x 4 block of radix-4 stages
        const int c1 = t & 15, r1 = t >> 4;
        uint2 rk[4];
        if (sa.slot) {
#pragma unroll
            for (int c2 = 0; c2 < 4; ++c2)
                rk[c2] = __ldg(reinterpret_cast<const uint2 *>(sa.rank + (size_t)j * MM +
                                                               ((size_t)((r1 & 7) * M + c1 + 16 * c2)) * 8));
        }
        {
            const float2 *w = sa.Wd ? sa.Wd + (size_t)sa.frame_sub[j] * MM : sa.w;
            const float2 *uj = sa.u + sa.frame_base[j];
            const int pitch = sa.frame_pitch[j];
            float2 x[4][4];
#pragma unroll
            for (int r2 = 0; r2 < 4; ++r2)
#pragma unroll
                for (int c2 = 0; c2 < 4; ++c2) {
                    const int row = r1 + 16 * r2, col = c1 + 16 * c2;
                    x[r2][c2] = cmul(__ldg(w + row * M + col), __ldg(uj + (size_t)row * pitch + col));
                }
#pragma unroll
            for (int c2 = 0; c2 < 4; ++c2) {
                float2 v[4] = {x[0][c2], x[1][c2], x[2][c2], x[3][c2]};
                dft<4, false>(v);
#pragma unroll
                for (int k1 = 0; k1 < 4; ++k1) x[k1][c2] = k1 ? cmul(v[k1], tw[r1 * k1]) : v[k1];
            }
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) {
                float2 v[4] = {x[k1][0], x[k1][1], x[k1][2], x[k1][3]};
                dft<4, false>(v);
#pragma unroll
                for (int l1 = 0; l1 < 4; ++l1)
                    buf[(16 * k1 + r1) * P + 16 * l1 + c1] = l1 ? cmul(v[l1], tw[c1 * l1]) : v[l1];
            }
        }
        __syncthreads();
        // ---- pass 2: column radix-16 over r1, in place
        {
            const int g = t & 63, k1 = t >> 6;
            float2 z[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) z[i] = buf[(16 * k1 + i) * P + g];
            dft<16, false>(z);
#pragma unroll
            for (int i = 0; i < 16; ++i) buf[(16 * k1 + i) * P + g] = z[i];
        }
        const bool ok = mbar_wait_bounded(bar, phase);
        if (__syncthreads_or(!ok)) {
            if (t == 0) *sa.err = 1;
            return;
        }
        phase ^= 1u;
        // ---- pass 3: row radix-16 over c1, prox and Gamma update, inverse row radix-16
        float rf = 0.f;
        {
            const int rho = t & 63, k = (rho >> 4) + 4 * (rho & 15), l1 = t >> 6, pk = pos64(k);
            float2 z[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) z[i] = buf[rho * P + 16 * l1 + i];
            float2 gmv[SG ? 1 : 16];
            if (!SG) {
#pragma unroll
                for (int l2 = 0; l2 < 16; ++l2)
                    gmv[SG ? 0 : l2] = sa.gamma[(size_t)j * MM + pos64(l1 + 4 * l2) * M + pk];
            }
            dft<16, false>(z);
#pragma unroll
            for (int l2 = 0; l2 < 16; ++l2) {
                const int li = pos64(l1 + 4 * l2) * M + pk;
                const float2 ax = cscale(z[l2], inv_m);  // (A_d u_d^n)_k
                const float sf = stg_f[li];
                const float2 gm = SG ? stg_g[li] : gmv[SG ? 0 : l2];
                const float a2 = ax.x * ax.x + ax.y * ax.y;
                rf += fabsf((a2 > 0.f ? a2 * rsqrtf(a2) : 0.f) - sf);  // | |A_d u_d| - sqrt f |
                const float2 y = cadd(gm, ax);                           // Gamma^n + A_d u_d^n
                const float2 zz = stagm_prox(y, sf, sa.pc);              // eq. updateZ
                const float2 gn = csub(y, zz);                           // eq. updateM-1-multi
                sa.gamma[(size_t)j * MM + li] = gn;
                z[l2] = csub(zz, gn);                                    // z^{n+1} - Gamma^{n+1}
            }
            dft<16, true>(z);
#pragma unroll
            for (int i = 0; i < 16; ++i) buf[rho * P + 16 * l1 + i] = z[i];
        }
        __syncthreads();  // staging buffers are free: start the next item's copies
        if (t == 0 && i + (int)gridDim.x < n_items) {
            fence_proxy_async_smem();
            issue(i + gridDim.x);
        }
        // ---- pass 4: inverse column radix-16, in place
        {
            const int g = t & 63, k1 = t >> 6;
            float2 z[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) z[i] = buf[(16 * k1 + i) * P + g];
            dft<16, true>(z);
#pragma unroll
            for (int i = 0; i < 16; ++i) buf[(16 * k1 + i) * P + g] = z[i];
        }
        __syncthreads();
        // ---- pass 5: inverse radix-4 stages, residual out
        {
            float2 x[4][4];
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) {
                float2 v[4];
#pragma unroll
                for (int l1 = 0; l1 < 4; ++l1) {
                    const float2 b = buf[(16 * k1 + r1) * P + 16 * l1 + c1];
                    v[l1] = l1 ? cmulc(b, tw[c1 * l1]) : b;
                }
                dft<4, true>(v);
#pragma unroll
                for (int c2 = 0; c2 < 4; ++c2) x[k1][c2] = k1 ? cmulc(v[c2], tw[r1 * k1]) : v[c2];
            }
#pragma unroll
            for (int c2 = 0; c2 < 4; ++c2) {
                float2 v[4] = {x[0][c2], x[1][c2], x[2][c2], x[3][c2]};
                dft<4, true>(v);
#pragma unroll
                for (int r2 = 0; r2 < 4; ++r2) x[r2][c2] = v[r2];
            }
            if (sa.slot) {
                // q_j = conj(w) o F^*(z - Gamma) into each pixel's gather slot
                const unsigned base = (unsigned)sa.frame_base[j], pitch = (unsigned)sa.frame_pitch[j];
#pragma unroll
                for (int r2 = 0; r2 < 4; ++r2)
#pragma unroll
                    for (int c2 = 0; c2 < 4; ++c2) {
                        const int row = r1 + 16 * r2, col = c1 + 16 * c2, b = (r1 >> 3) + 2 * r2;
                        const unsigned word = b < 4 ? rk[c2].x : rk[c2].y;
                        const unsigned rank = (word >> (8 * (b & 3))) & 0xffu;
                        const float2 v = cmulc(cscale(x[r2][c2], inv_m), __ldg(sa.w + row * M + col));
                        // 32-bit index: the plan checks slot_k * u_len < 2^32
                        sa.slot[rank * (unsigned)sa.slot_stride + base + (unsigned)row * pitch + (unsigned)col] = v;
                    }
            } else {
                // unweighted, natural order; the subdomain update weights with W_d^{n+1} (or w)
                float2 *o = sa.q + (size_t)j * MM;
#pragma unroll
                for (int r2 = 0; r2 < 4; ++r2)
#pragma unroll
                    for (int c2 = 0; c2 < 4; ++c2) o[(r1 + 16 * r2) * M + c1 + 16 * c2] = cscale(x[r2][c2], inv_m);
            }
        }
        // this frame's RF partial, one per warp (fixed xor tree inside the warp)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rf += __shfl_xor_sync(0xffffffffu, rf, o);
        if (lane == 0) sa.rf_part[j * (NT / 32) + warp] = rf;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- forward operator
template <int M>
__global__ void __launch_bounds__(Radix<M>::NT) forward_kernel(int J, const int32_t *base,
                                                                int pitch, const float2 *u,
                                                                const float2 *w, float2 *out,
                                                                const float2 *twg)
{
    constexpr int FPB = Radix<M>::FPB, NT = Radix<M>::NT, P = M + 1, MM = M * M;
    extern __shared__ float4 smem4[];
    float2 *tw = reinterpret_cast<float2 *>(smem4);
    float2 *buf = tw + M;
    const int j0 = blockIdx.x * FPB;
    for (int k = threadIdx.x; k < M; k += NT) tw[k] = twg[k];
    __syncthreads();
    constexpr int R1 = Radix<M>::R1, R2 = Radix<M>::R2;
    for (int task = threadIdx.x; task < FPB * M * R2; task += NT) {
        const int c = task % M, rest = task / M, n1 = rest % R2, f = rest / R2, j = j0 + f;
        if (j >= J) continue;
        const float2 *uj = u + base[j];
        float2 x[R1];
#pragma unroll
        for (int t = 0; t < R1; ++t) {
            const int row = n1 + R2 * t;
            x[t] = cmul(__ldg(w + row * M + c), __ldg(uj + (size_t)row * pitch + c));
        }
        dft<R1, false>(x);
        float2 *fb = buf + f * M * P;
#pragma unroll
        for (int s = 0; s < R1; ++s) fb[(n1 + R2 * s) * P + c] = cmul(x[s], tw[n1 * s]);
    }
    __syncthreads();
    col_stage2<M, false>(buf);
    __syncthreads();
    row_stage1<M, false>(buf, tw);
    __syncthreads();
    row_stage2<M, false>(buf);
    __syncthreads();
    const float inv_m = 1.f / (float)M;
    for (int e = threadIdx.x; e < FPB * MM; e += NT) {
        const int f = e / MM, k = e % MM, j = j0 + f;
        if (j >= J) continue;
        const int kr = k / M, kc = k % M;
        out[(size_t)j * MM + k] = cscale(buf[f * M * P + pos_of<M>(kr) * P + pos_of<M>(kc)], inv_m);
    }
}

// ---------------------------------------------------------------- frames -> F^* frames, x conj(w)
template <int M>
__global__ void __launch_bounds__(Radix<M>::NT) ifft_weight_kernel(int J, const float2 *in,
                                                                    const float2 *w, float2 *out,
                                                                    const float2 *twg)
{
    constexpr int FPB = Radix<M>::FPB, NT = Radix<M>::NT, P = M + 1, MM = M * M;
    extern __shared__ float4 smem4[];
    float2 *tw = reinterpret_cast<float2 *>(smem4);
    float2 *buf = tw + M;
    const int j0 = blockIdx.x * FPB;
    for (int k = threadIdx.x; k < M; k += NT) tw[k] = twg[k];
    for (int e = threadIdx.x; e < FPB * MM; e += NT) {
        const int f = e / MM, k = e % MM, j = j0 + f;
        if (j >= J) continue;
        buf[f * M * P + pos_of<M>(k / M) * P + pos_of<M>(k % M)] = __ldg(in + (size_t)j * MM + k);
    }
    __syncthreads();
    row_stage2<M, true>(buf);
    __syncthreads();
    row_stage1<M, true>(buf, tw);
    __syncthreads();
    col_stage2<M, true>(buf);
    __syncthreads();
    col_stage1_store<M>(buf, tw, j0, J, out, 1.f / (float)M, w);
}

// ---------------------------------------------------------------- loss frames
// h_j = F^* grad g(F(w o S_j u); f_j) (unweighted) and per-block loss partials.
// The exit wave reads the window at u + base[j] with row pitch `pitch`, or
// pitch_arr[j] when given (subdomain copies u_d), and the probe w, or
// Wd + frame_sub[j] * m^2 when Wd is given (blind subdomain probes).  With
// h = null only the loss partials are formed.
struct LossArgs {
    int32_t J, pitch;
    const int32_t *base, *pitch_arr, *frame_sub;
    const float2 *u, *w, *Wd;
    const float *sqrtf_;
    float2 *h;
    float *loss_part;
    const float2 *tw;
    float eps;
};

template <int M>
__global__ void __launch_bounds__(Radix<M>::NT) loss_kernel(LossArgs a)
{
    constexpr int R1 = Radix<M>::R1, R2 = Radix<M>::R2, FPB = Radix<M>::FPB, NT = Radix<M>::NT;
    constexpr int P = M + 1, MM = M * M;
    extern __shared__ float4 smem4[];
    float2 *tw = reinterpret_cast<float2 *>(smem4);
    float2 *buf = tw + M;
    float *red = reinterpret_cast<float *>(buf + FPB * M * P);
    const int j0 = blockIdx.x * FPB;
    if (threadIdx.x == 0) {  // this group's sqrt f into L2 while the forward FFT runs
        const unsigned bytes = (unsigned)(min(FPB, a.J - j0) * MM * sizeof(float));
        const char *fp = reinterpret_cast<const char *>(a.sqrtf_ + (size_t)j0 * MM);
        for (unsigned off = 0; off < bytes; off += 16384u) bulk_prefetch_l2(fp + off, min(16384u, bytes - off));
    }
    for (int k = threadIdx.x; k < M; k += NT) tw[k] = a.tw[k];
    __syncthreads();
    for (int task = threadIdx.x; task < FPB * M * R2; task += NT) {
        const int c = task % M, rest = task / M, n1 = rest % R2, f = rest / R2, j = j0 + f;
        if (j >= a.J) continue;
        const float2 *uj = a.u + a.base[j];
        const int pitch = a.pitch_arr ? a.pitch_arr[j] : a.pitch;
        const float2 *wj = a.Wd ? a.Wd + (size_t)a.frame_sub[j] * MM : a.w;
        float2 x[R1];
#pragma unroll
        for (int t = 0; t < R1; ++t) {
            const int row = n1 + R2 * t;
            x[t] = cmul(__ldg(wj + row * M + c), __ldg(uj + (size_t)row * pitch + c));
        }
        dft<R1, false>(x);
        float2 *fb = buf + f * M * P;
#pragma unroll
        for (int s = 0; s < R1; ++s) fb[(n1 + R2 * s) * P + c] = cmul(x[s], tw[n1 * s]);
    }
    __syncthreads();
    col_stage2<M, false>(buf);
    __syncthreads();
    row_stage1<M, false>(buf, tw);
    __syncthreads();
    float loss = 0.f;
    const float inv_m = 1.f / (float)M;
    const float eps = a.eps;
    const bool with_h = a.h != nullptr;  // the same for the whole block
    for (int task = threadIdx.x; task < FPB * M * R1; task += NT) {
        const int r = task % M, rest = task / M, s = rest % R1, f = rest / R1, j = j0 + f;
        if (j >= a.J) continue;
        float2 *fb = buf + f * M * P + r * P;
        float2 x[R2];
#pragma unroll
        for (int t = 0; t < R2; ++t) x[t] = fb[R2 * s + t];
        dft<R2, false>(x);
        const size_t base = (size_t)j * MM + r;
#pragma unroll
        for (int t = 0; t < R2; ++t) {
            const size_t idx = base + (size_t)(R2 * s + t) * M;
            const float2 xv = cscale(x[t], inv_m);
            const float sf = __ldg(a.sqrtf_ + idx);
            const float a2 = xv.x * xv.x + xv.y * xv.y;
            const float inv = rsqrtf(a2);  // 1/|x|, used only when a2 > 0
            const float ax = a2 > 0.f ? a2 * inv : 0.f;
            float gv, gs;  // g_eps (eq. obj-1) and grad g = gs * x (eq. objgrad)
            if (ax < eps * sf) {
                gv = 0.5f * (1.f - eps) * (sf * sf - a2 / eps);
                gs = 1.f - 1.f / eps;
            } else {
                gv = 0.5f * (ax - sf) * (ax - sf);
                gs = a2 > 0.f ? 1.f - sf * inv : 0.f;
            }
            loss += gv;
            x[t] = cscale(xv, gs);
        }
        if (with_h) {
            dft<R2, true>(x);
#pragma unroll
            for (int t = 0; t < R2; ++t) fb[R2 * s + t] = x[t];
        }
    }
    if (with_h) {
        __syncthreads();
        row_stage1<M, true>(buf, tw);
        __syncthreads();
        col_stage2<M, true>(buf);
        __syncthreads();
        col_stage1_store<M>(buf, tw, j0, a.J, a.h, inv_m, nullptr);
    }
    const float tot = block_sum_fixed(loss, red);
    if (threadIdx.x == 0) a.loss_part[blockIdx.x] = tot;
}

// ---------------------------------------------------------------- blind w-update (eq. blind_w)
// s * sum_d (Delta_d + W_d) per probe pixel (d ascending), all pixels in parallel.
__global__ void probe_sum_kernel(int MM, int D, const float2 *__restrict__ Wd, const float2 *__restrict__ Delta,
                                 float2 *__restrict__ out, float s)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= MM) return;
    float2 t = make_float2(0.f, 0.f);
    for (int d = 0; d < D; ++d) t = cadd(t, cadd(Delta[(size_t)d * MM + k], Wd[(size_t)d * MM + k]));
    out[k] = cscale(t, s);
}

// Masked probe average: w^{n+1} = (1/D) F^* M F sum, one block, from the sum
// that probe_sum_kernel left in wnew (in place).
template <int M>
__global__ void __launch_bounds__(Radix<M>::NT) probe_avg_kernel(int D, const float *mask, float2 *wnew,
                                                                  const float2 *twg)
{
    constexpr int NT = Radix<M>::NT, P = M + 1, MM = M * M;
    extern __shared__ float4 smem4[];
    float2 *tw = reinterpret_cast<float2 *>(smem4);
    float2 *buf = tw + M;
    const float invD = 1.f / (float)D;
    for (int k = threadIdx.x; k < M; k += NT) tw[k] = twg[k];
    for (int k = threadIdx.x; k < MM; k += NT) buf[(k / M) * P + (k % M)] = wnew[k];
    __syncthreads();
    col_stage1<M, false>(buf, tw);
    __syncthreads();
    col_stage2<M, false>(buf);
    __syncthreads();
    row_stage1<M, false>(buf, tw);
    __syncthreads();
    row_stage2<M, false>(buf);
    __syncthreads();
    // position (pr, pc) holds frequency (kr, kc); apply the support mask there
    for (int e = threadIdx.x; e < MM; e += NT) {
        const int pr = e / M, pc = e % M;
        const int kr = pr / Radix<M>::R2 + Radix<M>::R1 * (pr % Radix<M>::R2);
        const int kc = pc / Radix<M>::R2 + Radix<M>::R1 * (pc % Radix<M>::R2);
        buf[pr * P + pc] = cscale(buf[pr * P + pc], mask[kr * M + kc]);
    }
    __syncthreads();
    row_stage2<M, true>(buf);
    __syncthreads();
    row_stage1<M, true>(buf, tw);
    __syncthreads();
    col_stage2<M, true>(buf);
    __syncthreads();
    col_stage1<M, true>(buf, tw);
    __syncthreads();
    const float s = invD / (float)MM;  // two unitary 1/M factors and the 1/D average
    for (int k = threadIdx.x; k < MM; k += NT) wnew[k] = cscale(buf[(k / M) * P + (k % M)], s);
}

// ---------------------------------------------------------------- layout conversions
// f (natural) -> sqrt(max(f,0)) in transposed position layout; per-frame partial sums of sqrt f.
template <int M>
__global__ void ingest_f_kernel(int J, const float *f, float *sqrtf_, float *part)
{
    constexpr int MM = M * M;
    __shared__ float red[32];
    const int j = blockIdx.x;
    float acc = 0.f;
    for (int k = threadIdx.x; k < MM; k += blockDim.x) {
        const float v = sqrtf(fmaxf(__ldg(f + (size_t)j * MM + k), 0.f));
        sqrtf_[(size_t)j * MM + (size_t)pos_of<M>(k % M) * M + pos_of<M>(k / M)] = v;
        acc += v;
    }
    const float tot = block_sum_fixed(acc, red);
    if (threadIdx.x == 0) part[j] = tot;
}

template <int M>
__global__ void permute_kernel(int J, const float2 *src, float2 *dst, bool to_natural)
{
    constexpr int MM = M * M;
    const size_t n = (size_t)J * MM;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const size_t j = e / MM;
        const int k = (int)(e % MM);
        const size_t t = j * MM + (size_t)pos_of<M>(k % M) * M + pos_of<M>(k / M);
        if (to_natural)
            dst[e] = src[t];
        else
            dst[t] = src[e];
    }
}

constexpr int MAX_DEV = 64;     // per-device caches below are indexed by device ordinal
std::mutex g_attr_mu;            // guards every per-device attribute cache

// Raise a kernel's dynamic shared-memory limit once per device (the attribute
// belongs to the device's context).
template <int M, class K>
int set_smem(K kernel)
{
    static bool done[MAX_DEV] = {};
    int dev = 0;
    OD2P_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEV) return fail(PTYCHO_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (!done[dev]) {
        OD2P_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes<M>()));
        done[dev] = true;
    }
    return PTYCHO_OK;
}

// Runs the statement list with M_ (probe side) and V_ (launch shape) bound as
// compile-time constants for the shapes the frame update is compiled in.
#define OD2P_K1_SHAPE(m, v, ...)                                                   \
    switch ((m) * 2 + (v)) {                                                        \
    case 32: { constexpr int M_ = 16, V_ = 0; __VA_ARGS__; }                        \
    case 33: { constexpr int M_ = 16, V_ = 1; __VA_ARGS__; }                        \
    case 64: { constexpr int M_ = 32, V_ = 0; __VA_ARGS__; }                        \
    case 65: { constexpr int M_ = 32, V_ = 1; __VA_ARGS__; }                        \
    case 128: { constexpr int M_ = 64, V_ = 0; __VA_ARGS__; }                       \
    case 129: { constexpr int M_ = 64, V_ = 1; __VA_ARGS__; }                       \
    case 256: { constexpr int M_ = 128, V_ = 0; __VA_ARGS__; }                      \
    case 257: { constexpr int M_ = 128, V_ = 1; __VA_ARGS__; }                      \
    case 96: { constexpr int M_ = 48, V_ = 0; __VA_ARGS__; }                        \
    case 97: { constexpr int M_ = 48, V_ = 1; __VA_ARGS__; }                        \
    case 160: { constexpr int M_ = 80, V_ = 0; __VA_ARGS__; }                       \
    case 161: { constexpr int M_ = 80, V_ = 1; __VA_ARGS__; }                       \
    case 192: { constexpr int M_ = 96, V_ = 0; __VA_ARGS__; }                       \
    case 193: { constexpr int M_ = 96, V_ = 1; __VA_ARGS__; }                       \
    default: break;                                                                 \
    }

// Largest resident block count per SM of the frame update (both the single-plan
// and the batched instantiation), after raising its shared-memory limit.
template <int M, int V>
int k1_per_sm(int *per_sm_out, int *n_sm_out)
{
    static int per_sm[MAX_DEV] = {}, n_sm[MAX_DEV] = {};  // per device: the attribute is per context
    int dev = 0;
    OD2P_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEV) return fail(PTYCHO_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (!per_sm[dev]) {
        OD2P_CUDA(cudaFuncSetAttribute(frame_update_kernel<M, V, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)k1_smem_bytes<M, V>()));
        OD2P_CUDA(cudaFuncSetAttribute(frame_update_kernel<M, V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)k1_smem_bytes<M, V>()));
        int a = 0, b = 0, n = 0;
        OD2P_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        OD2P_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, frame_update_kernel<M, V, false>,
                                                                K1Cfg<M, V>::NT, k1_smem_bytes<M, V>()));
        OD2P_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, frame_update_kernel<M, V, true>,
                                                                K1Cfg<M, V>::NT, k1_smem_bytes<M, V>()));
        if (std::min(a, b) < 1) return fail(PTYCHO_ERR_UNSUPPORTED, "frame update does not fit on an SM");
        n_sm[dev] = n;
        per_sm[dev] = std::min(a, b);
    }
    *per_sm_out = per_sm[dev];
    *n_sm_out = n_sm[dev];
    return PTYCHO_OK;
}

template <int M, int V>
int frame_update_table_m(const FrameArgs *tab, const int2 *items, int n_items, int grid, int parity, cudaStream_t s)
{
    frame_update_kernel<M, V, true><<<grid, K1Cfg<M, V>::NT, k1_smem_bytes<M, V>(), s>>>(FrameArgs{}, tab, items,
                                                                                         n_items, parity);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

template <int M, int V>
int frame_update_single_m(const ptycho_plan_s *p, cudaStream_t s)
{
    const int groups = (p->J + K1Cfg<M, V>::FPB - 1) / K1Cfg<M, V>::FPB;
    frame_update_kernel<M, V, false><<<p->n_k1_blocks, K1Cfg<M, V>::NT, k1_smem_bytes<M, V>(), s>>>(
        p->h_fargs[p->cur], nullptr, nullptr, groups, p->cur);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

template <int M>
int forward_m(const ptycho_plan_s *p, const float2 *u, const float2 *w, float2 *out, cudaStream_t s)
{
    if (int rc = set_smem<M>(forward_kernel<M>)) return rc;
    const int blocks = (p->J + Radix<M>::FPB - 1) / Radix<M>::FPB;
    forward_kernel<M><<<blocks, Radix<M>::NT, smem_bytes<M>(), s>>>(p->J, p->d_img_base, p->img_cols, u, w,
                                                                     out, p->d_tw);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

template <int M>
int ifft_m(const ptycho_plan_s *p, const float2 *in, const float2 *w, float2 *out, cudaStream_t s)
{
    if (int rc = set_smem<M>(ifft_weight_kernel<M>)) return rc;
    const int blocks = (p->J + Radix<M>::FPB - 1) / Radix<M>::FPB;
    ifft_weight_kernel<M><<<blocks, Radix<M>::NT, smem_bytes<M>(), s>>>(p->J, in, w, out, p->d_tw);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

// subdomain = false: windows of the full image u (img_w pitch), probe w, and
// h_j to the plan's frame scratch; true: the plan's current subdomain copies
// u_d with their probes (W_d when blind), loss partials only.
template <int M>
int loss_m(ptycho_plan_s *p, const float2 *u, const float2 *w, cudaStream_t s, bool subdomain = false,
           float2 *h_out = nullptr)
{
    if (int rc = set_smem<M>(loss_kernel<M>)) return rc;
    LossArgs a;
    a.J = p->J;
    a.pitch = p->img_cols;
    a.base = subdomain ? p->d_frame_base : p->d_img_base;
    a.pitch_arr = subdomain ? p->d_frame_pitch : nullptr;
    a.frame_sub = p->d_frame_sub;
    a.u = u;
    a.w = w;
    a.Wd = subdomain && p->blind ? p->d_Wd : nullptr;
    a.sqrtf_ = p->d_sqrtf;
    a.h = subdomain ? nullptr : (h_out ? h_out : p->d_q);
    a.loss_part = p->d_loss_part;
    a.tw = p->d_tw;
    a.eps = p->eps;
    const int blocks = (p->J + Radix<M>::FPB - 1) / Radix<M>::FPB;
    loss_kernel<M><<<blocks, Radix<M>::NT, smem_bytes<M>(), s>>>(a);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

template <int M>
int probe_avg_m(ptycho_plan_s *p, cudaStream_t s)
{
    constexpr int MM = M * M;
    probe_sum_kernel<<<(MM + 255) / 256, 256, 0, s>>>(MM, p->D, p->d_Wd, p->d_Delta, p->d_wnew,
                                                       p->has_mask ? 1.f : 1.f / (float)p->D);
    OD2P_CUDA(cudaGetLastError());
    if (!p->has_mask) return PTYCHO_OK;
    probe_avg_kernel<M><<<1, Radix<M>::NT, smem_bytes<M>(), s>>>(p->D, p->d_mask, p->d_wnew, p->d_tw);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

template <int M>
int ingest_m(ptycho_plan_s *p, const float *f, float *part, cudaStream_t s)
{
    ingest_f_kernel<M><<<p->J, 256, 0, s>>>(p->J, f, p->d_sqrtf, part);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

template <int M>
int permute_m(const ptycho_plan_s *p, const float2 *src, float2 *dst, bool to_nat, cudaStream_t s)
{
    const size_t n = (size_t)p->J * M * M;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
    permute_kernel<M><<<blocks, 256, 0, s>>>(p->J, src, dst, to_nat);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

}  // namespace

bool supported_m(int m)
{
    return m == 16 || m == 32 || m == 64 || m == 128 || m == 256 || m == 48 || m == 80 || m == 96;
}

void rank_radix(int m, int *R1, int *R2)
{
    switch (m) {
    case 16: *R1 = Radix<16>::R1, *R2 = Radix<16>::R2; break;
    case 32: *R1 = Radix<32>::R1, *R2 = Radix<32>::R2; break;
    case 64: *R1 = Radix<64>::R1, *R2 = Radix<64>::R2; break;
    case 128: *R1 = Radix<128>::R1, *R2 = Radix<128>::R2; break;
    case 48: *R1 = Radix<48>::R1, *R2 = Radix<48>::R2; break;
    case 80: *R1 = Radix<80>::R1, *R2 = Radix<80>::R2; break;
    case 96: *R1 = Radix<96>::R1, *R2 = Radix<96>::R2; break;
    default: *R1 = *R2 = 0; break;
    }
}

int frames_per_block(int m)
{
    switch (m) {
    case 16: return Radix<16>::FPB;
    case 32: return Radix<32>::FPB;
    case 64: return Radix<64>::FPB;
    case 128: return Radix<128>::FPB;
    case 48: return Radix<48>::FPB;
    case 80: return Radix<80>::FPB;
    case 96: return Radix<96>::FPB;
    default: return 1;
    }
}

// Blocks of the persistent frame update for n_items frame groups of side m,
// launch shape `variant`, at most blocks_per_sm (0: as many as fit) per SM;
// max_per_sm (optional) receives the most that fit.
int frame_update_grid(int m, int variant, int n_items, int blocks_per_sm, int *grid, int *max_per_sm)
{
    if (m == 256) {
        *grid = n_items;
        if (max_per_sm) *max_per_sm = 1;
        return PTYCHO_OK;
    }
    int per_sm = 0, n_sm = 0, rc = PTYCHO_ERR_UNSUPPORTED;
    OD2P_K1_SHAPE(m, variant, rc = k1_per_sm<M_, V_>(&per_sm, &n_sm); break)
    if (rc) return rc == PTYCHO_ERR_UNSUPPORTED ? fail(rc, "probe side m must be 16, 32, 48, 64, 80, 96, 128 or 256") : rc;
    if (max_per_sm) *max_per_sm = per_sm;
    const int bps = blocks_per_sm > 0 ? std::min(blocks_per_sm, per_sm) : per_sm;
    *grid = std::max(1, std::min(n_items, bps * n_sm));
    return PTYCHO_OK;
}

namespace {
template <int M>
int prepare_m()
{
    int per_sm = 0, n_sm = 0;
    if (int rc = k1_per_sm<M, 0>(&per_sm, &n_sm)) return rc;
    if (int rc = k1_per_sm<M, 1>(&per_sm, &n_sm)) return rc;
    if (int rc = set_smem<M>(forward_kernel<M>)) return rc;
    if (int rc = set_smem<M>(ifft_weight_kernel<M>)) return rc;
    if (int rc = set_smem<M>(loss_kernel<M>)) return rc;
    return set_smem<M>(probe_avg_kernel<M>);
}
}  // namespace

// Raise the dynamic shared-memory limit of every frame kernel of size m once,
// outside any stream capture.
int prepare_kernels(int m)
{
    switch (m) {
    case 16: return prepare_m<16>();
    case 32: return prepare_m<32>();
    case 64: return prepare_m<64>();
    case 128: return prepare_m<128>();
    case 48: return prepare_m<48>();
    case 80: return prepare_m<80>();
    case 96: return prepare_m<96>();
    case 256: return PTYCHO_OK;  // its kernels stay within the default shared-memory limit
    default: return fail(PTYCHO_ERR_UNSUPPORTED, "probe side m must be 16, 32, 48, 64, 80, 96, 128 or 256");
    }
}

// Frame groups of the frame update (m <= 128) or 16-column slabs (m = 256).
int frame_groups(int m, int J, int variant)
{
    OD2P_K1_SHAPE(m, variant, return (J + K1Cfg<M_, V_>::FPB - 1) / K1Cfg<M_, V_>::FPB)
    return J * 16;
}

// RF partial sums written per iteration: one per warp of each frame group
// (m <= 128); m = 256: one per 16-column slab of the column pass (variant 0)
// or per CTA of a frame's cluster (variant 1).
int rf_parts(int m, int J, int variant)
{
    OD2P_K1_SHAPE(m, variant, return frame_groups(m, J, variant) * (K1Cfg<M_, V_>::NT / 32))
    return rf_parts_256(J, variant);
}

void fill_frame_args(const ptycho_plan_s *p, FrameArgs out[2])
{
    for (int par = 0; par < 2; ++par) {
        FrameArgs &a = out[par];
        a = FrameArgs{};
        a.J = p->J;
        a.frame_sub = p->d_frame_sub;
        a.frame_base = p->d_frame_base;
        a.frame_pitch = p->d_frame_pitch;
        a.u = p->d_u[par];
        a.w = p->d_w;
        a.Wd = p->blind ? p->d_Wd : nullptr;
        a.gamma = p->d_gamma;
        a.sqrtf_ = p->d_sqrtf;
        a.q = p->d_q;
        a.slot = p->slots ? p->d_slot : nullptr;
        a.rank = p->d_rank;
        a.slot_stride = (int32_t)p->u_len;
        a.rf_part = p->d_rf_part;
        a.err = p->d_err;
        a.tw = p->d_tw;
        a.pc = make_prox_const(p->eps, p->eta);
    }
}

int launch_frame_update_table(int m, int variant, const FrameArgs *tab, const int2 *items, int n_items, int grid,
                              int parity, cudaStream_t s)
{
    OD2P_K1_SHAPE(m, variant, return frame_update_table_m<M_, V_>(tab, items, n_items, grid, parity, s))
    return fail(PTYCHO_ERR_UNSUPPORTED, "table-driven frame update: m must be at most 128");
}

// The 16 x 4 split for m = 64 (fft kinds 1 and 2): blocks that fit per SM
// (after raising the shared-memory limit once per device) and the launch.
template <int SG>
int f4_per_sm(int *per_sm_out, int *n_sm_out)
{
    static int per_sm[MAX_DEV] = {}, n_sm[MAX_DEV] = {};
    int dev = 0;
    OD2P_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEV) return fail(PTYCHO_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (!per_sm[dev]) {
        OD2P_CUDA(cudaFuncSetAttribute(frame_update_f4_kernel<SG, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)f4_smem_bytes<SG>()));
        OD2P_CUDA(cudaFuncSetAttribute(frame_update_f4_kernel<SG, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)f4_smem_bytes<SG>()));
        int a = 0, n = 0;
        OD2P_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        OD2P_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, frame_update_f4_kernel<SG, true>, F4Cfg<SG>::NT,
                                                                f4_smem_bytes<SG>()));
        if (a < 1) return fail(PTYCHO_ERR_UNSUPPORTED, "the 16 x 4 frame update does not fit on an SM");
        per_sm[dev] = a;
        n_sm[dev] = n;
    }
    *per_sm_out = per_sm[dev];
    *n_sm_out = n_sm[dev];
    return PTYCHO_OK;
}

int f4_grid(int kind, int J, int *grid, int blocks_per_sm)
{
    int per_sm = 0, n_sm = 0;
    if (int rc = kind == 1 ? f4_per_sm<1>(&per_sm, &n_sm) : f4_per_sm<0>(&per_sm, &n_sm)) return rc;
    const int bps = blocks_per_sm > 0 ? std::min(blocks_per_sm, per_sm) : per_sm;
    *grid = std::max(1, std::min(J, bps * n_sm));
    return PTYCHO_OK;
}

// The batches' m = 64 class on the 16 x 4 split (fft kind 2): one persistent
// launch over the members' (plan, frame) items.
int launch_frame_update_f4_table(const FrameArgs *tab, const int2 *items, int n_items, int grid, int parity,
                                 cudaStream_t s)
{
    int per_sm = 0, n_sm = 0;
    if (int rc = f4_per_sm<0>(&per_sm, &n_sm)) return rc;  // the shared-memory limit, once per device
    if (n_items <= 0) return PTYCHO_OK;
    frame_update_f4_kernel<0, true><<<grid, 256, f4_smem_bytes<0>(), s>>>(FrameArgs{}, tab, items, n_items, parity);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_frame_update(ptycho_plan_s *p, cudaStream_t s)
{
    if (p->M == 256) return frame_update_256(p, s);
    if (p->fft_kind) {
        if (p->fft_kind == 1)
            frame_update_f4_kernel<1, false><<<p->n_k1_blocks, 256, f4_smem_bytes<1>(), s>>>(
                p->h_fargs[p->cur], nullptr, nullptr, p->J, 0);
        else
            frame_update_f4_kernel<0, false><<<p->n_k1_blocks, 256, f4_smem_bytes<0>(), s>>>(
                p->h_fargs[p->cur], nullptr, nullptr, p->J, 0);
        OD2P_CUDA(cudaGetLastError());
        return PTYCHO_OK;
    }
    OD2P_K1_SHAPE(p->M, p->k1_variant, return frame_update_single_m<M_, V_>(p, s))
    switch (p->M) {
    default: return fail(PTYCHO_ERR_UNSUPPORTED, "probe side m must be 16, 32, 48, 64, 80, 96, 128 or 256");
    }
}

int launch_forward(const ptycho_plan_s *p, const float2 *u, const float2 *w, float2 *out, cudaStream_t s)
{
    switch (p->M) {
    case 16: return forward_m<16>(p, u, w, out, s);
    case 32: return forward_m<32>(p, u, w, out, s);
    case 64: return forward_m<64>(p, u, w, out, s);
    case 128: return forward_m<128>(p, u, w, out, s);
    case 48: return forward_m<48>(p, u, w, out, s);
    case 80: return forward_m<80>(p, u, w, out, s);
    case 96: return forward_m<96>(p, u, w, out, s);
    case 256: return forward_256(p, u, w, out, s);
    default: return fail(PTYCHO_ERR_UNSUPPORTED, "probe side m must be 16, 32, 48, 64, 80, 96, 128 or 256");
    }
}

int launch_frames_ifft_weight(const ptycho_plan_s *p, const float2 *frames, const float2 *w,
                              bool ifft, float2 *out, cudaStream_t s)
{
    if (!ifft) return fail(PTYCHO_ERR_STATE, "internal: spatial frames need no transform");
    switch (p->M) {
    case 16: return ifft_m<16>(p, frames, w, out, s);
    case 32: return ifft_m<32>(p, frames, w, out, s);
    case 64: return ifft_m<64>(p, frames, w, out, s);
    case 128: return ifft_m<128>(p, frames, w, out, s);
    case 48: return ifft_m<48>(p, frames, w, out, s);
    case 80: return ifft_m<80>(p, frames, w, out, s);
    case 96: return ifft_m<96>(p, frames, w, out, s);
    case 256:
        if (w) return fail(PTYCHO_ERR_STATE, "internal: m = 256 inverse FFT takes no weight");
        return ifft_256(p, frames, out, s);
    default: return fail(PTYCHO_ERR_UNSUPPORTED, "probe side m must be 16, 32, 48, 64, 80, 96, 128 or 256");
    }
}

int launch_loss_frames(ptycho_plan_s *p, const float2 *u, const float2 *w, cudaStream_t s, float2 *h_out)
{
    switch (p->M) {
    case 16: return loss_m<16>(p, u, w, s, false, h_out);
    case 32: return loss_m<32>(p, u, w, s, false, h_out);
    case 64: return loss_m<64>(p, u, w, s, false, h_out);
    case 128: return loss_m<128>(p, u, w, s, false, h_out);
    case 48: return loss_m<48>(p, u, w, s, false, h_out);
    case 80: return loss_m<80>(p, u, w, s, false, h_out);
    case 96: return loss_m<96>(p, u, w, s, false, h_out);
    case 256: return loss_256(p, u, w, s, h_out);
    default: return fail(PTYCHO_ERR_UNSUPPORTED, "probe side m must be 16, 32, 48, 64, 80, 96, 128 or 256");
    }
}

int launch_metrics_loss(ptycho_plan_s *p, cudaStream_t s)
{
    const float2 *u = p->d_u[p->cur];
    switch (p->M) {
    case 16: return loss_m<16>(p, u, p->d_w, s, true);
    case 32: return loss_m<32>(p, u, p->d_w, s, true);
    case 64: return loss_m<64>(p, u, p->d_w, s, true);
    case 128: return loss_m<128>(p, u, p->d_w, s, true);
    case 48: return loss_m<48>(p, u, p->d_w, s, true);
    case 80: return loss_m<80>(p, u, p->d_w, s, true);
    case 96: return loss_m<96>(p, u, p->d_w, s, true);
    case 256: return loss_256_sub(p, s);
    default: return fail(PTYCHO_ERR_UNSUPPORTED, "probe side m must be 16, 32, 48, 64, 80, 96, 128 or 256");
    }
}

int launch_probe_avg(ptycho_plan_s *p, cudaStream_t s)
{
    switch (p->M) {
    case 16: return probe_avg_m<16>(p, s);
    case 32: return probe_avg_m<32>(p, s);
    case 64: return probe_avg_m<64>(p, s);
    case 128: return probe_avg_m<128>(p, s);
    case 48: return probe_avg_m<48>(p, s);
    case 80: return probe_avg_m<80>(p, s);
    case 96: return probe_avg_m<96>(p, s);
    case 256: return probe_avg_256(p, s);
    default: return fail(PTYCHO_ERR_UNSUPPORTED, "probe side m must be 16, 32, 48, 64, 80, 96, 128 or 256");
    }
}

int launch_ingest_f(ptycho_plan_s *p, const float *f, cudaStream_t s)
{
    float *part = p->d_loss_part;  // J floats of scratch, reduced in launch_sum_sqrtf
    switch (p->M) {
    case 16: return ingest_m<16>(p, f, part, s);
    case 32: return ingest_m<32>(p, f, part, s);
    case 64: return ingest_m<64>(p, f, part, s);
    case 128: return ingest_m<128>(p, f, part, s);
    case 48: return ingest_m<48>(p, f, part, s);
    case 80: return ingest_m<80>(p, f, part, s);
    case 96: return ingest_m<96>(p, f, part, s);
    case 256: return ingest_256(p, f, part, s);
    default: return fail(PTYCHO_ERR_UNSUPPORTED, "probe side m must be 16, 32, 48, 64, 80, 96, 128 or 256");
    }
}

int launch_permute_gamma(const ptycho_plan_s *p, const float2 *src, float2 *dst, bool to_natural,
                         cudaStream_t s)
{
    switch (p->M) {
    case 16: return permute_m<16>(p, src, dst, to_natural, s);
    case 32: return permute_m<32>(p, src, dst, to_natural, s);
    case 64: return permute_m<64>(p, src, dst, to_natural, s);
    case 128: return permute_m<128>(p, src, dst, to_natural, s);
    case 48: return permute_m<48>(p, src, dst, to_natural, s);
    case 80: return permute_m<80>(p, src, dst, to_natural, s);
    case 96: return permute_m<96>(p, src, dst, to_natural, s);
    case 256: return permute_256(p, src, dst, to_natural, s);
    default: return fail(PTYCHO_ERR_UNSUPPORTED, "probe side m must be 16, 32, 48, 64, 80, 96, 128 or 256");
    }
}

}  // namespace od2p

// ---------------------------------------------------------------- allocation-free loss
// stagm_loss_noalloc: the loss part of stagm_loss_grad without a plan and
// without any device allocation.  Its only scratch -- one partial sum per
// block -- is the file-scope array below, which every GPU that loads this
// library holds for the life of the process.
namespace od2p {
namespace {

constexpr int NOALLOC_MAX_BLOCKS = 65536;  // 256 KiB of partial sums
__device__ __align__(256) float g_noalloc_partials[NOALLOC_MAX_BLOCKS];

// Host-side device addresses of g_noalloc_partials, one per device, filled by
// the first call on that device (the symbol's host name is not an address).
constexpr int NOALLOC_MAX_DEVICES = 64;
float *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
bool g_noalloc_attr[NOALLOC_MAX_DEVICES][4] = {};  // shared-memory limit raised, per m
std::mutex g_noalloc_mu;

struct NoallocArgs {
    int32_t J, H, W;
    const int32_t *offs;
    const float2 *u, *w;
    const float *f;  // natural frequency order
    float *partials;
    float eps;
};

template <int M>
__global__ void __launch_bounds__(Radix<M>::NT) loss_noalloc_kernel(NoallocArgs a)
{
    constexpr int R1 = Radix<M>::R1, R2 = Radix<M>::R2, FPB = Radix<M>::FPB, NT = Radix<M>::NT;
    constexpr int P = M + 1, MM = M * M;
    extern __shared__ float4 smem4[];
    float2 *tw = reinterpret_cast<float2 *>(smem4);
    float2 *buf = tw + M;
    float *red = reinterpret_cast<float *>(buf + FPB * M * P);
    __shared__ int bad_window;
    const int j0 = blockIdx.x * FPB;
    if (threadIdx.x == 0) bad_window = 0;
    // twiddles exp(-2 pi i k / M) from the exact single-precision routine
    for (int k = threadIdx.x; k < M; k += NT) {
        float sn, cs;
        sincospif(-2.f * (float)k / (float)M, &sn, &cs);
        tw[k] = make_float2(cs, sn);
    }
    __syncthreads();
    for (int task = threadIdx.x; task < FPB * M * R2; task += NT) {
        const int c = task % M, rest = task / M, n1 = rest % R2, f = rest / R2, j = j0 + f;
        if (j >= a.J) continue;
        const int r0 = __ldg(a.offs + 2 * j), c0 = __ldg(a.offs + 2 * j + 1);
        float2 x[R1];
        if (r0 < 0 || c0 < 0 || r0 > a.H - M || c0 > a.W - M) {
            // a window outside the image: no load, and the block's partial becomes NaN
            bad_window = 1;
#pragma unroll
            for (int t = 0; t < R1; ++t) x[t] = make_float2(0.f, 0.f);
        } else {
            const float2 *uj = a.u + (size_t)r0 * a.W + c0;
#pragma unroll
            for (int t = 0; t < R1; ++t) {
                const int row = n1 + R2 * t;
                x[t] = cmul(__ldg(a.w + row * M + c), __ldg(uj + (size_t)row * a.W + c));
            }
        }
        dft<R1, false>(x);
        float2 *fb = buf + f * M * P;
#pragma unroll
        for (int s = 0; s < R1; ++s) fb[(n1 + R2 * s) * P + c] = cmul(x[s], tw[n1 * s]);
    }
    __syncthreads();
    col_stage2<M, false>(buf);
    __syncthreads();
    row_stage1<M, false>(buf, tw);
    __syncthreads();
    float loss = 0.f;
    const float inv_m = 1.f / (float)M, eps = a.eps;
    for (int task = threadIdx.x; task < FPB * M * R1; task += NT) {
        const int r = task % M, rest = task / M, s = rest % R1, f = rest / R1, j = j0 + f;
        if (j >= a.J) continue;
        float2 *fb = buf + f * M * P + r * P;
        float2 x[R2];
#pragma unroll
        for (int t = 0; t < R2; ++t) x[t] = fb[R2 * s + t];
        dft<R2, false>(x);
        const int kr = r / R2 + R1 * (r % R2);
#pragma unroll
        for (int t = 0; t < R2; ++t) {
            const int pc = R2 * s + t, kc = pc / R2 + R1 * (pc % R2);
            const float sf = sqrtf(fmaxf(__ldg(a.f + (size_t)j * MM + kr * M + kc), 0.f));
            const float2 xv = cscale(x[t], inv_m);
            const float ax = sqrtf(xv.x * xv.x + xv.y * xv.y);
            loss += ax < eps * sf ? 0.5f * (1.f - eps) * (sf * sf - ax * ax / eps)
                                  : 0.5f * (ax - sf) * (ax - sf);
        }
    }
    const float tot = block_sum_fixed(loss, red);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = bad_window ? __int_as_float(0x7fc00000) : tot;
}

// Sum of the n partials in a fixed order: each thread a contiguous run, then warps in order.
__global__ void __launch_bounds__(256) noalloc_sum_kernel(int n, const float *partials, float *out)
{
    __shared__ double red[8];
    const int per = (n + 255) / 256;
    double t = 0.0;
    for (int i = threadIdx.x * per; i < min(n, (threadIdx.x + 1) * per); ++i) t += partials[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < 8; ++i) s += red[i];
        *out = (float)s;
    }
}

// Raises the kernel's dynamic shared-memory limit on the current device; the
// caller holds g_noalloc_mu and records success only after this returns OK.
template <int M>
int noalloc_setup_m()
{
    OD2P_CUDA(cudaFuncSetAttribute(loss_noalloc_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem_bytes<M>()));
    return PTYCHO_OK;
}

template <int M>
int loss_noalloc_m(const NoallocArgs &base, float *loss, cudaStream_t s)
{
    const int blocks = (base.J + Radix<M>::FPB - 1) / Radix<M>::FPB;
    if (blocks > NOALLOC_MAX_BLOCKS)
        return fail(PTYCHO_ERR_INVALID_ARG,
                    "stagm_loss_noalloc: at most " + std::to_string((long long)NOALLOC_MAX_BLOCKS * Radix<M>::FPB) +
                        " frames of side " + std::to_string(M) + " (fixed scratch)");
    loss_noalloc_kernel<M><<<blocks, Radix<M>::NT, smem_bytes<M>(), s>>>(base);
    OD2P_CUDA(cudaGetLastError());
    noalloc_sum_kernel<<<1, 256, 0, s>>>(blocks, base.partials, loss);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

}  // namespace
}  // namespace od2p

extern "C" int stagm_loss_noalloc(const ptycho_c32 *u, int32_t img_h, int32_t img_w, const ptycho_c32 *w,
                                  int32_t m, const int32_t *offsets_dev, int32_t n_frames, const float *f,
                                  float eps, float *loss, ptycho_stream_t stream)
{
    using namespace od2p;
    if (!u || !w || !offsets_dev || !f || !loss) return fail(PTYCHO_ERR_INVALID_ARG, "NULL argument");
    if (!(m == 16 || m == 32 || m == 64 || m == 128))
        return fail(PTYCHO_ERR_UNSUPPORTED, "stagm_loss_noalloc: probe side m must be 16, 32, 64 or 128");
    if (n_frames < 1 || img_h < m || img_w < m) return fail(PTYCHO_ERR_INVALID_ARG, "need n_frames >= 1 and an image at least m x m");
    if (!(eps > 0.f && eps < 1.f)) return fail(PTYCHO_ERR_INVALID_ARG, "eps must be in (0, 1)");
    // per-device set-up: the device address of the file-scope scratch array
    int dev = 0;
    OD2P_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(PTYCHO_ERR_UNSUPPORTED, "device index out of range");
    const int mi = m == 16 ? 0 : m == 32 ? 1 : m == 64 ? 2 : 3;
    float *scratch;
    {
        // per-device, per-m set-up under the lock; a flag is set only once its
        // step has succeeded, so a failed step is retried by the next call and no
        // thread launches before the shared-memory limit has been raised
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *ptr = nullptr;
            OD2P_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_partials));
            g_noalloc_ptr[dev] = static_cast<float *>(ptr);
        }
        if (!g_noalloc_attr[dev][mi]) {
            const int rc = m == 16 ? noalloc_setup_m<16>() : m == 32 ? noalloc_setup_m<32>()
                         : m == 64 ? noalloc_setup_m<64>() : noalloc_setup_m<128>();
            if (rc != PTYCHO_OK) return rc;
            g_noalloc_attr[dev][mi] = true;
        }
        scratch = g_noalloc_ptr[dev];
    }
    NoallocArgs a;
    a.J = n_frames;
    a.H = img_h;
    a.W = img_w;
    a.offs = offsets_dev;
    a.u = reinterpret_cast<const float2 *>(u);
    a.w = reinterpret_cast<const float2 *>(w);
    a.f = f;
    a.partials = scratch;
    a.eps = eps;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (m) {
    case 16: return loss_noalloc_m<16>(a, loss, s);
    case 32: return loss_noalloc_m<32>(a, loss, s);
    case 64: return loss_noalloc_m<64>(a, loss, s);
    default: return loss_noalloc_m<128>(a, loss, s);
    }
}
