// Frame-space kernels for probe side m = 256.
//
// A 256 x 256 complex64 frame is 512 KB, more than one block's shared memory,
// so its unitary 2-D FFT runs as three passes over frame slabs:
//   A: 16-row slabs -- exit wave (or a plain frame), row FFTs (16 x 16 DIF);
//   B: 16-column slabs -- column FFTs, the elementwise step of the caller
//      (ST-AGM prox + Gamma update, loss and gradient, Fourier mask, or output),
//      then the inverse column FFTs;
//   C: 16-row slabs -- inverse row FFTs, natural-order output.
// The intermediate T (natural rows / position columns after A, the reverse
// after B) is a plan-owned buffer of WAVE frames: frames go through A, B, C in
// waves of WAVE frames (512 KB each), so T stays in L2 between the passes and HBM sees the
// algorithmic traffic plus q.  Position p = 16 s + s' holds frequency s + 16 s'
// along each axis (as for the smaller sizes); Gamma and sqrt f are stored at
// position row-major index p_r * 256 + p_c.
#include "od2p_internal.h"
#include "fft_device.cuh"

#include <mutex>

namespace od2p {
namespace {

constexpr int BM = 256, BR = 16, BMM = BM * BM;
constexpr int SLAB = 16;   // rows (A, C) or columns (B) per block
constexpr int NTB = 256;   // threads per block
constexpr int PA = BM + 1; // pitch of a row slab in shared memory
constexpr int PB = SLAB + 1;

__device__ __forceinline__ int freq_of(int p) { return p / BR + BR * (p % BR); }

enum ModeB : int { B_PROX = 0, B_FWD_OUT = 1, B_LOSS = 2, B_MASK = 3, B_IFFT_IN = 4 };

struct PassA {
    int32_t j0, nf;
    const int32_t *frame_sub, *frame_base, *frame_pitch;  // exit-wave source
    const float2 *u, *w, *Wd;
    const float2 *plain;  // plain-frame source (natural spatial), or null
    float2 *T;
    const float2 *tw;
};

struct PassB {
    int32_t j0, nf, mode;
    float2 *T;
    float2 *gamma;
    const float *sqrtf_;
    const float2 *in;   // B_IFFT_IN: natural-frequency frames
    float2 *out;        // B_FWD_OUT: natural-frequency frames
    const float *mask;  // B_MASK: natural-frequency support
    float *part;        // per-block partial sums (RF or loss)
    int32_t part_off;
    const float2 *tw;
    ProxConst pc;
    float eps;
};

struct PassC {
    int32_t j0, nf;
    const float2 *T;
    float2 *out;
    const float2 *wconj;  // optional: multiply the output by conj(wconj)
    float scale;
    // optional: write into the nonblind gather slots instead of `out`
    float2 *slot;
    const uint8_t *rank;
    const int32_t *frame_base, *frame_pitch;
    int32_t slot_stride;
};

__global__ void __launch_bounds__(NTB) rows_fwd256_kernel(PassA a)
{
    extern __shared__ float4 smem4[];
    float2 *tw = reinterpret_cast<float2 *>(smem4);
    float2 *buf = tw + BM;
    const int f = blockIdx.x / (BM / SLAB), rb = blockIdx.x % (BM / SLAB), j = a.j0 + f;
    for (int k = threadIdx.x; k < BM; k += NTB) tw[k] = a.tw[k];
    const int c = threadIdx.x;
    // all of the thread's loads in flight before the first shared-memory store
    float2 v[SLAB];
    if (a.plain) {
#pragma unroll
        for (int r = 0; r < SLAB; ++r) v[r] = __ldg(a.plain + (size_t)j * BMM + (rb * SLAB + r) * BM + c);
    } else {
        const float2 *w = a.Wd ? a.Wd + (size_t)a.frame_sub[j] * BMM : a.w;
        const float2 *uj = a.u + a.frame_base[j];
        const int pitch = a.frame_pitch[j];
        float2 wv[SLAB];
#pragma unroll
        for (int r = 0; r < SLAB; ++r) {
            const int row = rb * SLAB + r;
            wv[r] = __ldg(w + row * BM + c);
            v[r] = __ldg(uj + (size_t)row * pitch + c);
        }
#pragma unroll
        for (int r = 0; r < SLAB; ++r) v[r] = cmul(wv[r], v[r]);
    }
#pragma unroll
    for (int r = 0; r < SLAB; ++r) buf[r * PA + c] = v[r];
    __syncthreads();
    {   // row stage 1: lanes on rows (odd pitch), 16 strided elements each
        const int r = threadIdx.x % SLAB, n1 = threadIdx.x / SLAB;
        float2 *rp = buf + r * PA;
        float2 x[BR];
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = rp[n1 + BR * t];
        dft<BR, false>(x);
#pragma unroll
        for (int s = 0; s < BR; ++s) rp[n1 + BR * s] = cmul(x[s], tw[n1 * s]);
    }
    __syncthreads();
    {   // row stage 2: 16 contiguous elements
        const int r = threadIdx.x % SLAB, s = threadIdx.x / SLAB;
        float2 *rp = buf + r * PA + BR * s;
        float2 x[BR];
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = rp[t];
        dft<BR, false>(x);
#pragma unroll
        for (int t = 0; t < BR; ++t) rp[t] = x[t];
    }
    __syncthreads();
    for (int r = 0; r < SLAB; ++r) a.T[((size_t)f * BM + rb * SLAB + r) * BM + c] = buf[r * PA + c];
}

#ifndef OD2P_COLS256_MINB
#define OD2P_COLS256_MINB 4
#endif
// MODE: the elementwise step between the column transforms (compile-time, so
// that the per-element loop carries no mode tests).
template <int MODE>
__global__ void __launch_bounds__(NTB, OD2P_COLS256_MINB) cols256_kernel(PassB a)
{
    extern __shared__ float4 smem4[];
    float2 *tw = reinterpret_cast<float2 *>(smem4);
    float2 *buf = tw + BM;                       // BM rows x PB
    float *red = reinterpret_cast<float *>(buf + BM * PB);
    const int f = blockIdx.x / (BM / SLAB), cb = blockIdx.x % (BM / SLAB), j = a.j0 + f;
    if (MODE == B_PROX) {
        // this slab's Gamma (128 B) and sqrt f (64 B) of each position row, into
        // L2 while the column FFT runs
        const size_t gi = (size_t)j * BMM + (size_t)threadIdx.x * BM + cb * SLAB;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.gamma + gi));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.sqrtf_ + gi));
    }
    for (int k = threadIdx.x; k < BM; k += NTB) tw[k] = a.tw[k];
    {
        constexpr int NR = BM / (NTB / SLAB);  // rows per thread
        const int cl = threadIdx.x % SLAB, r0 = threadIdx.x / SLAB;
        float2 v[NR];
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            const int r = r0 + i * (NTB / SLAB);
            if (MODE == B_IFFT_IN)
                v[i] = __ldg(a.in + (size_t)j * BMM + freq_of(r) * BM + freq_of(cb * SLAB + cl));
            else
                v[i] = a.T[((size_t)f * BM + r) * BM + cb * SLAB + cl];
        }
#pragma unroll
        for (int i = 0; i < NR; ++i) buf[(r0 + i * (NTB / SLAB)) * PB + cl] = v[i];
    }
    __syncthreads();
    const int cl = threadIdx.x % SLAB, hi = threadIdx.x / SLAB;  // hi: n1 (stage 1) or s (stage 2)
    if (MODE != B_IFFT_IN) {  // column stage 1
        float2 x[BR];
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = buf[(hi + BR * t) * PB + cl];
        dft<BR, false>(x);
#pragma unroll
        for (int s = 0; s < BR; ++s) buf[(hi + BR * s) * PB + cl] = cmul(x[s], tw[hi * s]);
        __syncthreads();
    }
    float part = 0.f;
    {   // column stage 2, the elementwise step, inverse column stage 2
        float2 x[BR];
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = buf[(BR * hi + t) * PB + cl];
        const int pc = cb * SLAB + cl;
        // this thread's column segment of Gamma and sqrt f (position rows
        // 16 hi .. 16 hi + 15), loaded before any Gamma store (the compiler may
        // not move loads past those stores)
        const size_t g0 = (size_t)j * BMM + (size_t)(BR * hi) * BM + pc;
        float2 *gseg = a.gamma + g0;
        const float *fseg = a.sqrtf_ + g0;
        float2 gmv[MODE == B_PROX ? BR : 1];
        float sfv[MODE == B_PROX || MODE == B_LOSS ? BR : 1];
        if (MODE == B_PROX || MODE == B_LOSS) {
#pragma unroll
            for (int t = 0; t < BR; ++t) {
                // read once per iteration: streaming loads (evict first) keep the
                // intermediate T resident in L2
                sfv[t] = __ldcs(fseg + t * BM);
                if (MODE == B_PROX) gmv[MODE == B_PROX ? t : 0] = __ldcs(gseg + t * BM);
            }
        }
        if (MODE != B_IFFT_IN) dft<BR, false>(x);
        const float inv_m = 1.f / (float)BM;
#pragma unroll
        for (int t = 0; t < BR; ++t) {
            const int pr = BR * hi + t;
            const size_t gi = (size_t)j * BMM + (size_t)pr * BM + pc;
            if (MODE == B_PROX) {
                const float2 ax = cscale(x[t], inv_m);
                const float sf = sfv[t];
                const float2 gm = gmv[MODE == B_PROX ? t : 0];
                const float a2 = ax.x * ax.x + ax.y * ax.y;
                part += fabsf((a2 > 0.f ? a2 * rsqrtf(a2) : 0.f) - sf);
                const float2 y = cadd(gm, ax);
                const float2 z = stagm_prox(y, sf, a.pc);
                const float2 gn = csub(y, z);
                __stcs(gseg + t * BM, gn);
                x[t] = csub(z, gn);
            } else if (MODE == B_LOSS) {
                const float2 xv = cscale(x[t], inv_m);
                const float sf = sfv[MODE == B_LOSS ? t : 0];
                const float ax = sqrtf(xv.x * xv.x + xv.y * xv.y);
                float gs;
                if (ax < a.eps * sf) {
                    part += 0.5f * (1.f - a.eps) * (sf * sf - ax * ax / a.eps);
                    gs = 1.f - 1.f / a.eps;
                } else {
                    part += 0.5f * (ax - sf) * (ax - sf);
                    gs = ax > 0.f ? 1.f - sf / ax : 0.f;
                }
                x[t] = cscale(xv, gs);
            } else if (MODE == B_MASK) {
                x[t] = cscale(x[t], inv_m * __ldg(a.mask + freq_of(pr) * BM + freq_of(pc)));
            } else if (MODE == B_FWD_OUT) {
                a.out[(size_t)j * BMM + freq_of(pr) * BM + freq_of(pc)] = cscale(x[t], inv_m);
            }
        }
        if (MODE != B_FWD_OUT) {
            dft<BR, true>(x);
#pragma unroll
            for (int t = 0; t < BR; ++t) buf[(BR * hi + t) * PB + cl] = x[t];
        }
    }
    if (MODE == B_PROX || MODE == B_LOSS) {
        const float tot = block_sum_fixed(part, red);
        if (threadIdx.x == 0) a.part[a.part_off + blockIdx.x] = tot;
    }
    if (MODE == B_FWD_OUT) return;
    __syncthreads();
    {   // inverse column stage 1
        float2 x[BR];
#pragma unroll
        for (int s = 0; s < BR; ++s) x[s] = cmulc(buf[(hi + BR * s) * PB + cl], tw[hi * s]);
        dft<BR, true>(x);
#pragma unroll
        for (int t = 0; t < BR; ++t) buf[(hi + BR * t) * PB + cl] = x[t];
    }
    __syncthreads();
    {
        const int c2 = threadIdx.x % SLAB, r0 = threadIdx.x / SLAB;
        for (int r = r0; r < BM; r += NTB / SLAB)
            a.T[((size_t)f * BM + r) * BM + cb * SLAB + c2] = buf[r * PB + c2];
    }
}

__global__ void __launch_bounds__(NTB) rows_inv256_kernel(PassC a, const float2 *twg)
{
    extern __shared__ float4 smem4[];
    float2 *tw = reinterpret_cast<float2 *>(smem4);
    float2 *buf = tw + BM;
    const int f = blockIdx.x / (BM / SLAB), rb = blockIdx.x % (BM / SLAB), j = a.j0 + f;
    for (int k = threadIdx.x; k < BM; k += NTB) tw[k] = twg[k];
    const int c = threadIdx.x;
    {
        float2 v[SLAB];
#pragma unroll
        for (int r = 0; r < SLAB; ++r) v[r] = a.T[((size_t)f * BM + rb * SLAB + r) * BM + c];
#pragma unroll
        for (int r = 0; r < SLAB; ++r) buf[r * PA + c] = v[r];
    }
    __syncthreads();
    {   // inverse row stage 2
        const int r = threadIdx.x % SLAB, s = threadIdx.x / SLAB;
        float2 *rp = buf + r * PA + BR * s;
        float2 x[BR];
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = rp[t];
        dft<BR, true>(x);
#pragma unroll
        for (int t = 0; t < BR; ++t) rp[t] = x[t];
    }
    __syncthreads();
    {   // inverse row stage 1
        const int r = threadIdx.x % SLAB, n1 = threadIdx.x / SLAB;
        float2 *rp = buf + r * PA;
        float2 x[BR];
#pragma unroll
        for (int s = 0; s < BR; ++s) x[s] = cmulc(rp[n1 + BR * s], tw[n1 * s]);
        dft<BR, true>(x);
#pragma unroll
        for (int t = 0; t < BR; ++t) rp[n1 + BR * t] = x[t];
    }
    __syncthreads();
    // the output rows rb * SLAB .. of column c, with the mode tests and the
    // per-frame bases hoisted out of the row loop
    const float sc = a.scale;
    const size_t r0 = (size_t)rb * SLAB;
    if (a.slot) {  // nonblind gather slots: conj(w) o q_j at the pixel's rank
        const int pitch = a.frame_pitch[j];
        const uint8_t *rk = a.rank + (size_t)j * BMM + r0 * BM + c;
        const float2 *wc = a.wconj + r0 * BM + c;
        float2 *sl = a.slot + a.frame_base[j] + r0 * pitch + c;
        const size_t stride = (size_t)a.slot_stride;
#pragma unroll
        for (int r = 0; r < SLAB; ++r)
            sl[__ldg(rk + r * BM) * stride + (size_t)r * pitch] = cmulc(cscale(buf[r * PA + c], sc), __ldg(wc + r * BM));
    } else {
        float2 *o = a.out + (size_t)j * BMM + r0 * BM + c;
        if (a.wconj) {
            const float2 *wc = a.wconj + r0 * BM + c;
#pragma unroll
            for (int r = 0; r < SLAB; ++r) o[r * BM] = cmulc(cscale(buf[r * PA + c], sc), __ldg(wc + r * BM));
        } else {
#pragma unroll
            for (int r = 0; r < SLAB; ++r) __stcs(o + r * BM, cscale(buf[r * PA + c], sc));
        }
    }
}

// ---------------------------------------------------------------- single-pass frame update
// One thread-block cluster of CL CTAs holds one 256 x 256 frame in its
// distributed shared memory, so the frame crosses HBM once per direction and
// no intermediate leaves the chip.  CTA c of the cluster owns rows
// [RPC c, RPC c + RPC) of the frame while the rows are transformed (buffer A)
// and position columns [CPC c, CPC c + CPC) while the columns are (buffer B).
// Between the phases every CTA sends each part of its data to the CTA that
// owns it next with asynchronous shared-memory stores into that CTA's other
// buffer (st.async), each completing bytes on the receiver's transaction
// barrier; a CTA proceeds once its barrier has counted all the bytes it is
// owed.  Sending into the buffer the receiver is not reading needs no barrier
// across the cluster: a CTA sends only values computed from what it has read.
// The arithmetic is that of passes A, B and C above, operation for operation
// (the same 16 x 16 splits, twiddles, prox and scaling); with CL = 16 a CTA's
// columns are one column slab of pass B with the same thread mapping, so its
// RF partial (one per CTA) is grouped as pass B's.  Every barrier wait is
// bounded; a wait that gives up sets the plan's device error flag.
__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_arrive_relaxed()
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait()
{
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
// shared::cluster address of shared::cta address `a` in CTA `rank`
__device__ __forceinline__ unsigned cluster_addr(unsigned a, unsigned rank)
{
    unsigned out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(a), "r"(rank));
    return out;
}
__device__ __forceinline__ void st_async_v4(unsigned addr, float4 v, unsigned bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     addr),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void st_async_v2(unsigned addr, float2 v, unsigned bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(addr),
                 "f"(v.x), "f"(v.y), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void tbar_expect(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// wait for phase 0 of a transaction barrier; false after 2^22 polls
__device__ __forceinline__ bool tbar_wait(uint64_t *bar)
{
    for (int i = 0; i < (1 << 22); ++i) {
        unsigned ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok)
                     : "r"(smem_addr(bar))
                     : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void prefetch_bulk_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

#ifndef OD2P_CL256
#define OD2P_CL256 16
#endif
template <int CL>
struct Cl256 {
    static constexpr int RPC = BM / CL;  // rows per CTA in the row phase
    static constexpr int CPC = BM / CL;  // position columns per CTA in the column phase
    static constexpr int NT = BR * RPC;  // one 16-point DFT per thread and stage
    static constexpr int MINB = 768 / NT;
    static constexpr int PR = BM + 1;    // buffer A pitch (odd: conflict-free stage-2 reads)
    static constexpr int PC = CPC + 2;   // buffer B pitch (16-byte rows, spread banks)
    static constexpr int A_ELEMS = RPC * PR, B_ELEMS = BM * PC;
    static constexpr unsigned XBYTES = (unsigned)(BM * CPC * sizeof(float2));  // bytes owed per exchange
    static constexpr size_t SMEM = sizeof(float2) * (BM + A_ELEMS + B_ELEMS) + 2 * sizeof(uint64_t) +
                                   sizeof(float) * (NT / 32);
};

template <int CL>
__global__ void __launch_bounds__(Cl256<CL>::NT, Cl256<CL>::MINB) frame_update256_cluster_kernel(FrameArgs a)
{
    using K = Cl256<CL>;
    constexpr int RPC = K::RPC, CPC = K::CPC, NT = K::NT, PR = K::PR, PC = K::PC;
    static_assert(RPC * 16 * CL == BM * 16 && K::XBYTES == (unsigned)(RPC * BM * sizeof(float2)), "layout");
    extern __shared__ float4 smem4[];
    float2 *tw = reinterpret_cast<float2 *>(smem4);
    float2 *bufA = tw + BM;           // rows RPC c ..: RPC x PR
    float2 *bufB = bufA + K::A_ELEMS;  // position columns CPC c ..: BM x PC
    uint64_t *bar = reinterpret_cast<uint64_t *>(bufB + K::B_ELEMS);  // [0]: columns owed, [1]: rows owed
    float *red = reinterpret_cast<float *>(bar + 2);
    const int tid = threadIdx.x;
    const unsigned c = cluster_rank();
    const int j = blockIdx.x / CL;
    const size_t fo = (size_t)j * BMM;
    if (tid == 0) {
        tbar_init(&bar[0]);
        tbar_init(&bar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // every CTA's barriers are initialised before any CTA sends to them (waited
    // for just before the first send)
    cluster_arrive_relaxed();
    // this CTA's Gamma and sqrt f columns of every position row, into L2 while
    // the row transforms run
    for (int k = tid; k < 2 * BM; k += NT) {
        const size_t gi = fo + (size_t)(k % BM) * BM + CPC * c;
        if (k < BM)
            prefetch_bulk_l2(a.gamma + gi, CPC * sizeof(float2));
        else
            prefetch_bulk_l2(a.sqrtf_ + gi, CPC * sizeof(float));
    }
    for (int k = tid; k < BM; k += NT) tw[k] = a.tw[k];
    // ---- rows, stage 1: exit wave w o S_j u of row RPC c + r, DFTs over t at n1
    {
        const int n1 = tid % BR, r = tid / BR, row = RPC * c + r;
        const float2 *w = (a.Wd ? a.Wd + (size_t)a.frame_sub[j] * BMM : a.w) + row * BM + n1;
        const float2 *uj = a.u + a.frame_base[j] + (size_t)row * a.frame_pitch[j] + n1;
        float2 x[BR];
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = cmul(__ldg(w + BR * t), __ldg(uj + BR * t));
        dft<BR, false>(x);
        __syncthreads();  // twiddles in place
        float2 *rp = bufA + r * PR;
#pragma unroll
        for (int s = 0; s < BR; ++s) rp[n1 + BR * s] = cmul(x[s], tw[n1 * s]);
    }
    __syncthreads();
    // ---- rows, stage 2: DFTs over n1 -> positions 16 s + k; first exchange
    {
        const int r = tid % RPC, s = tid / RPC;
        float2 x[BR];
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = bufA[r * PR + BR * s + t];
        dft<BR, false>(x);
        if (tid == 0) tbar_expect(&bar[0], K::XBYTES);
        cluster_wait();  // the receivers' barriers are initialised
        // position columns 16 s .. 16 s + 15 of row RPC c + r belong to CTA 16 s / CPC
        const unsigned dst = (unsigned)(BR * s) / CPC;
        const unsigned da = cluster_addr(smem_addr(bufB + (RPC * c + r) * PC + (BR * s) % CPC), dst);
        const unsigned db = cluster_addr(smem_addr(&bar[0]), dst);
#pragma unroll
        for (int k = 0; k < BR / 2; ++k)
            st_async_v4(da + 16u * k, make_float4(x[2 * k].x, x[2 * k].y, x[2 * k + 1].x, x[2 * k + 1].y), db);
    }
    if (!tbar_wait(&bar[0])) *a.err = 1;  // every CTA's share of this CTA's columns has arrived
    // ---- columns, stage 1: DFTs over t at n1 of position column CPC c + col
    {
        const int col = tid % CPC, n1 = tid / CPC;
        float2 x[BR];
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = bufB[(n1 + BR * t) * PC + col];
        dft<BR, false>(x);
#pragma unroll
        for (int s = 0; s < BR; ++s) bufB[(n1 + BR * s) * PC + col] = cmul(x[s], tw[n1 * s]);
    }
    __syncthreads();
    // ---- columns, stage 2, the ST-AGM prox and Gamma update (eqs. updateZ,
    // updateM-1-multi) on position rows 16 s + t, inverse stage 2
    float part = 0.f;
    {
        const int col = tid % CPC, s = tid / CPC, pc = CPC * c + col;
        float2 x[BR];
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = bufB[(BR * s + t) * PC + col];
        float2 gmv[BR];
        float sfv[BR];
        const float2 *gp = a.gamma + fo + (size_t)(BR * s) * BM + pc;
        const float *fp = a.sqrtf_ + fo + (size_t)(BR * s) * BM + pc;
#pragma unroll
        for (int t = 0; t < BR; ++t) {
            sfv[t] = __ldg(fp + t * BM);
            gmv[t] = gp[t * BM];
        }
        dft<BR, false>(x);
        const float inv_m = 1.f / (float)BM;
        float2 *gw = a.gamma + fo + (size_t)(BR * s) * BM + pc;
#pragma unroll
        for (int t = 0; t < BR; ++t) {
            const float2 ax = cscale(x[t], inv_m);
            const float sf = sfv[t];
            const float a2 = ax.x * ax.x + ax.y * ax.y;
            part += fabsf((a2 > 0.f ? a2 * rsqrtf(a2) : 0.f) - sf);
            const float2 y = cadd(gmv[t], ax);
            const float2 z = stagm_prox(y, sf, a.pc);
            const float2 gn = csub(y, z);
            gw[t * BM] = gn;
            x[t] = csub(z, gn);
        }
        dft<BR, true>(x);
#pragma unroll
        for (int t = 0; t < BR; ++t) bufB[(BR * s + t) * PC + col] = x[t];
    }
    __syncthreads();
    // ---- columns, inverse stage 1 -> spatial rows n1 + 16 t; second exchange
    {
        const int col = tid % CPC, n1 = tid / CPC, pc = CPC * c + col;
        float2 x[BR];
#pragma unroll
        for (int s = 0; s < BR; ++s) x[s] = cmulc(bufB[(n1 + BR * s) * PC + col], tw[n1 * s]);
        dft<BR, true>(x);
        if (tid == 0) tbar_expect(&bar[1], K::XBYTES);
#pragma unroll
        for (int t = 0; t < BR; ++t) {
            const int R = n1 + BR * t;  // spatial row, owned by CTA R / RPC
            const unsigned dst = (unsigned)(R / RPC);
            st_async_v2(cluster_addr(smem_addr(bufA + (R % RPC) * PR + pc), dst), x[t],
                        cluster_addr(smem_addr(&bar[1]), dst));
        }
    }
    if (!tbar_wait(&bar[1])) *a.err = 1;  // this CTA's rows have arrived
    // ---- rows, inverse stage 2
    {
        const int r = tid % RPC, s = tid / RPC;
        float2 *rp = bufA + r * PR + BR * s;
        float2 x[BR];
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = rp[t];
        dft<BR, true>(x);
#pragma unroll
        for (int t = 0; t < BR; ++t) rp[t] = x[t];
    }
    __syncthreads();
    // ---- rows, inverse stage 1 -> spatial columns n1 + 16 t; q_j, or conj(w) q_j
    // into the gather slots (nonblind)
    {
        const int n1 = tid % BR, r = tid / BR, row = RPC * c + r;
        const float2 *rp = bufA + r * PR;
        float2 x[BR];
#pragma unroll
        for (int s = 0; s < BR; ++s) x[s] = cmulc(rp[n1 + BR * s], tw[n1 * s]);
        dft<BR, true>(x);
        const float sc = 1.f / (float)BM;
        if (a.slot) {
            const uint8_t *rk = a.rank + fo + row * BM + n1;
            float2 *sl = a.slot + a.frame_base[j] + (size_t)row * a.frame_pitch[j] + n1;
#pragma unroll
            for (int t = 0; t < BR; ++t) {
                const float2 v = cmulc(cscale(x[t], sc), __ldg(a.w + row * BM + n1 + BR * t));
                sl[(size_t)__ldg(rk + BR * t) * a.slot_stride + BR * t] = v;
            }
        } else {
            float2 *q = a.q + fo + row * BM + n1;
#pragma unroll
            for (int t = 0; t < BR; ++t) q[BR * t] = cscale(x[t], sc);
        }
    }
    const float tot = block_sum_fixed(part, red);
    if (tid == 0) a.rf_part[(size_t)j * CL + c] = tot;
    // no CTA leaves while stores of its cluster may still be in flight
    cluster_arrive_relaxed();
    cluster_wait();
}

int cluster256_setup(const void *fn, size_t smem)
{
    static bool done[64] = {};
    static std::mutex mu;
    int dev = 0;
    OD2P_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(PTYCHO_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(mu);
    if (!done[dev]) {
        OD2P_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        OD2P_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        done[dev] = true;
    }
    return PTYCHO_OK;
}

int frame_update_256_cluster(ptycho_plan_s *p, cudaStream_t s)
{
    using K = Cl256<OD2P_CL256>;
    auto fn = frame_update256_cluster_kernel<OD2P_CL256>;
    if (int rc = cluster256_setup(reinterpret_cast<const void *>(fn), K::SMEM)) return rc;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)p->J * OD2P_CL256);
    cfg.blockDim = dim3(K::NT);
    cfg.dynamicSmemBytes = K::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = OD2P_CL256;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    OD2P_CUDA(cudaLaunchKernelEx(&cfg, fn, p->h_fargs[p->cur]));
    return PTYCHO_OK;
}

constexpr size_t SMEM_A = sizeof(float2) * (BM + SLAB * PA);
constexpr size_t SMEM_B = sizeof(float2) * (BM + BM * PB) + sizeof(float) * (NTB / 32);

// One pass-A / pass-B / pass-C sequence over frames [j0, j0 + J) in waves.
struct Pipeline {
    bool do_a, do_c;
    PassA A;
    PassB B;
    PassC C;
};

int run_waves(Pipeline P, int J, int waves_frames, cudaStream_t s)
{
    const int slabs = BM / SLAB;
    for (int w0 = 0; w0 < J; w0 += waves_frames) {
        const int nf = std::min(waves_frames, J - w0);
        if (P.do_a) {
            PassA a = P.A;
            a.j0 = w0;
            a.nf = nf;
            rows_fwd256_kernel<<<nf * slabs, NTB, SMEM_A, s>>>(a);
            OD2P_CUDA(cudaGetLastError());
        }
        PassB b = P.B;
        b.j0 = w0;
        b.nf = nf;
        b.part_off = w0 * slabs;
        switch (b.mode) {
        case B_PROX: cols256_kernel<B_PROX><<<nf * slabs, NTB, SMEM_B, s>>>(b); break;
        case B_FWD_OUT: cols256_kernel<B_FWD_OUT><<<nf * slabs, NTB, SMEM_B, s>>>(b); break;
        case B_LOSS: cols256_kernel<B_LOSS><<<nf * slabs, NTB, SMEM_B, s>>>(b); break;
        case B_MASK: cols256_kernel<B_MASK><<<nf * slabs, NTB, SMEM_B, s>>>(b); break;
        default: cols256_kernel<B_IFFT_IN><<<nf * slabs, NTB, SMEM_B, s>>>(b); break;
        }
        OD2P_CUDA(cudaGetLastError());
        if (P.do_c) {
            PassC c = P.C;
            c.j0 = w0;
            c.nf = nf;
            rows_inv256_kernel<<<nf * slabs, NTB, SMEM_A, s>>>(c, P.B.tw);
            OD2P_CUDA(cudaGetLastError());
        }
    }
    return PTYCHO_OK;
}

Pipeline base_pipeline(const ptycho_plan_s *p)
{
    Pipeline P{};
    P.A.frame_sub = p->d_frame_sub;
    P.A.frame_base = p->d_frame_base;
    P.A.frame_pitch = p->d_frame_pitch;
    P.A.T = p->d_T;
    P.A.tw = p->d_tw;
    P.B.T = p->d_T;
    P.B.tw = p->d_tw;
    P.B.gamma = p->d_gamma;
    P.B.sqrtf_ = p->d_sqrtf;
    P.B.pc = make_prox_const(p->eps, p->eta);
    P.B.eps = p->eps;
    P.C.T = p->d_T;
    return P;
}

__global__ void ingest256_kernel(int J, const float *f, float *sqrtf_, float *part)
{
    __shared__ float red[32];
    const int j = blockIdx.x;
    float acc = 0.f;
    for (int k = threadIdx.x; k < BMM; k += blockDim.x) {
        const int kr = k / BM, kc = k % BM;
        const int pr = BR * (kr % BR) + kr / BR, pc = BR * (kc % BR) + kc / BR;
        const float v = sqrtf(fmaxf(__ldg(f + (size_t)j * BMM + k), 0.f));
        sqrtf_[(size_t)j * BMM + pr * BM + pc] = v;
        acc += v;
    }
    const float tot = block_sum_fixed(acc, red);
    if (threadIdx.x == 0) part[j] = tot;
}

__global__ void permute256_kernel(int J, const float2 *src, float2 *dst, bool to_natural)
{
    const size_t n = (size_t)J * BMM;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const size_t j = e / BMM;
        const int k = (int)(e % BMM), kr = k / BM, kc = k % BM;
        const size_t t = j * BMM + (size_t)(BR * (kr % BR) + kr / BR) * BM + (BR * (kc % BR) + kc / BR);
        if (to_natural)
            dst[e] = src[t];
        else
            dst[t] = src[e];
    }
}

__global__ void probe_sum256_kernel(int D, const float2 *Wd, const float2 *Delta, float2 *out, float scale)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= BMM) return;
    float2 t = make_float2(0.f, 0.f);
    for (int d = 0; d < D; ++d) t = cadd(t, cadd(Delta[(size_t)d * BMM + k], Wd[(size_t)d * BMM + k]));
    out[k] = cscale(t, scale);
}

}  // namespace

int rf_parts_256(int J, int variant) { return variant == 1 ? J * OD2P_CL256 : J * (BM / SLAB); }

int frame_update_256(ptycho_plan_s *p, cudaStream_t s)
{
    if (p->k1_variant == 1) return frame_update_256_cluster(p, s);
    Pipeline P = base_pipeline(p);
    P.do_a = P.do_c = true;
    P.A.u = p->d_u[p->cur];
    P.A.w = p->d_w;
    P.A.Wd = p->blind ? p->d_Wd : nullptr;
    P.B.mode = B_PROX;
    P.B.part = p->d_rf_part;
    P.C.out = p->d_q;
    P.C.wconj = p->slots ? p->d_w : nullptr;
    P.C.scale = 1.f / (float)BM;
    if (p->slots) {
        P.C.slot = p->d_slot;
        P.C.rank = p->d_rank;
        P.C.frame_base = p->d_frame_base;
        P.C.frame_pitch = p->d_frame_pitch;
        P.C.slot_stride = (int32_t)p->u_len;
    }
    return run_waves(P, p->J, WAVE_256, s);
}

int forward_256(const ptycho_plan_s *p, const float2 *u, const float2 *w, float2 *out, cudaStream_t s)
{
    Pipeline P = base_pipeline(p);
    P.do_a = true;
    P.do_c = false;
    P.A.frame_base = p->d_img_base;  // windows of the full image: pitch img_w
    P.A.frame_pitch = p->d_img_pitch;
    P.A.u = u;
    P.A.w = w;
    P.B.mode = B_FWD_OUT;
    P.B.out = out;
    return run_waves(P, p->J, WAVE_256, s);
}

int ifft_256(const ptycho_plan_s *p, const float2 *in, float2 *out, cudaStream_t s)
{
    Pipeline P = base_pipeline(p);
    P.do_a = false;
    P.do_c = true;
    P.B.mode = B_IFFT_IN;
    P.B.in = in;
    P.C.out = out;
    P.C.scale = 1.f / (float)BM;
    return run_waves(P, p->J, WAVE_256, s);
}

int loss_256(ptycho_plan_s *p, const float2 *u, const float2 *w, cudaStream_t s, float2 *h_out)
{
    Pipeline P = base_pipeline(p);
    P.do_a = P.do_c = true;
    P.A.frame_base = p->d_img_base;
    P.A.frame_pitch = p->d_img_pitch;
    P.A.u = u;
    P.A.w = w;
    P.B.mode = B_LOSS;
    P.B.part = p->d_loss_part;
    P.C.out = h_out ? h_out : p->d_q;
    P.C.scale = 1.f / (float)BM;
    return run_waves(P, p->J, WAVE_256, s);
}

int loss_256_sub(ptycho_plan_s *p, cudaStream_t s)
{
    Pipeline P = base_pipeline(p);
    P.do_a = true;
    P.do_c = false;
    P.A.u = p->d_u[p->cur];
    P.A.w = p->d_w;
    P.A.Wd = p->blind ? p->d_Wd : nullptr;
    P.B.mode = B_LOSS;
    P.B.part = p->d_loss_part;
    return run_waves(P, p->J, WAVE_256, s);
}

int probe_avg_256(ptycho_plan_s *p, cudaStream_t s)
{
    const float invD = 1.f / (float)p->D;
    if (!p->has_mask) {
        probe_sum256_kernel<<<BMM / 256, 256, 0, s>>>(p->D, p->d_Wd, p->d_Delta, p->d_wnew, invD);
        OD2P_CUDA(cudaGetLastError());
        return PTYCHO_OK;
    }
    // sum into wave slot 0 of T, then F^* M F in place, scaled by 1/D on the way out
    probe_sum256_kernel<<<BMM / 256, 256, 0, s>>>(p->D, p->d_Wd, p->d_Delta, p->d_T, 1.f);
    OD2P_CUDA(cudaGetLastError());
    Pipeline P = base_pipeline(p);
    P.do_a = P.do_c = true;
    P.A.plain = p->d_T;
    P.B.mode = B_MASK;
    P.B.mask = p->d_mask;
    P.C.out = p->d_wnew;
    P.C.scale = invD / (float)BM;
    return run_waves(P, 1, 1, s);
}

int ingest_256(ptycho_plan_s *p, const float *f, float *part, cudaStream_t s)
{
    ingest256_kernel<<<p->J, 256, 0, s>>>(p->J, f, p->d_sqrtf, part);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int permute_256(const ptycho_plan_s *p, const float2 *src, float2 *dst, bool to_natural, cudaStream_t s)
{
    const size_t n = (size_t)p->J * BMM;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
    permute256_kernel<<<blocks, 256, 0, s>>>(p->J, src, dst, to_natural);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

}  // namespace od2p
