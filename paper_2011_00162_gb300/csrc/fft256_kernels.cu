// Frame-space kernels for probe side m = 256.
//
// A 256 x 256 complex64 frame is 512 KB, more than one block's shared memory,
// so its unitary 2-D FFT runs as three passes over frame slabs:
//   A: 16-row slabs -- exit wave (or a plain frame), row FFTs;
//   B: 16-column slabs -- column FFTs, the elementwise step of the caller
//      (ST-AGM prox + Gamma update, loss and gradient, Fourier mask, or output),
//      then the inverse column FFTs;
//   C: 16-row slabs -- inverse row FFTs, natural-order output.
// Every 256-point transform is 16 x 16: with n = n1 + 16 n2 and k = k1 + 16 k2,
// stage 1 takes a 16-point DFT over n2 at fixed n1, the twiddle
// exp(-+2 pi i n1 k1 / 256), and stage 2 a 16-point DFT over n1 at fixed k1.
// A thread that holds the elements n1 + 16 n2 of a row (stage 1) or the
// frequencies k1 + 16 k2 (stage 2 output) reads or writes them straight from
// or to global memory, sixteen lanes covering 128 contiguous bytes, so each
// pass exchanges data through shared memory once per transform direction.
// The intermediate T (spatial rows / frequency columns after A, the reverse
// after B) is a plan-owned buffer per wave chain: frames go through A, B, C in
// waves (512 KB a frame), so T stays in L2 between the passes and HBM sees the
// algorithmic traffic plus q.  T, Gamma and sqrt f hold frequencies in natural
// row-major order (k_r * 256 + k_c).
#include "od2p_internal.h"
#include "fft_device.cuh"

#include <mutex>

namespace od2p {
namespace {

constexpr int BM = 256, BR = 16, BMM = BM * BM;
constexpr int SLAB = 16;   // rows (A, C) or columns (B) per block
constexpr int NTB = 256;   // threads per block
constexpr int PX = BR * (BR + 1);  // pitch of a row in a row slab: 16 groups of 17
constexpr int PB = SLAB + 1;
static_assert(NTB * 128 == SLAB * BM * (int)sizeof(float2), "pass C: one 128-byte L2 line of its slab per thread");

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
    float2 *buf = tw + BM;  // SLAB rows x PX: stage-1 output (k1, n1) at 17 k1 + n1
    const int f = blockIdx.x / (BM / SLAB), rb = blockIdx.x % (BM / SLAB), j = a.j0 + f;
    for (int k = threadIdx.x; k < BM; k += NTB) tw[k] = a.tw[k];
    // thread (r, lo): stage 1 at n1 = lo, stage 2 at k1 = lo; sixteen lanes
    // touch 128 contiguous bytes of one row in every global access
    const int lo = threadIdx.x % BR, r = threadIdx.x / BR, row = rb * SLAB + r;
    float2 x[BR];
    if (a.plain) {
        const float2 *src = a.plain + (size_t)j * BMM + row * BM + lo;
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = __ldg(src + BR * t);
    } else {
        const float2 *w = (a.Wd ? a.Wd + (size_t)a.frame_sub[j] * BMM : a.w) + row * BM + lo;
        const float2 *uj = a.u + a.frame_base[j] + (size_t)row * a.frame_pitch[j] + lo;
        float2 wv[BR];
#pragma unroll
        for (int t = 0; t < BR; ++t) {
            wv[t] = __ldg(w + BR * t);
            x[t] = __ldg(uj + BR * t);
        }
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = cmul(wv[t], x[t]);
    }
    // row stage 1: DFT over n2 of the elements n1 + 16 n2
    dft<BR, false>(x);
    __syncthreads();  // twiddles in place
    float2 *rp = buf + r * PX;
#pragma unroll
    for (int s = 0; s < BR; ++s) rp[(BR + 1) * s + lo] = cmul(x[s], tw[lo * s]);
    __syncthreads();
    // row stage 2: DFT over n1 -> frequencies k1 + 16 k2, stored in natural order
#pragma unroll
    for (int t = 0; t < BR; ++t) x[t] = rp[(BR + 1) * lo + t];
    dft<BR, false>(x);
    float2 *o = a.T + ((size_t)f * BM + row) * BM + lo;
#pragma unroll
    for (int t = 0; t < BR; ++t) o[BR * t] = x[t];
}

#ifndef OD2P_COLS256_MINB
#define OD2P_COLS256_MINB 3
#endif
// MODE: the elementwise step between the column transforms (compile-time, so
// that the per-element loop carries no mode tests).
template <int MODE>
__global__ void __launch_bounds__(NTB, OD2P_COLS256_MINB) cols256_kernel(PassB a)
{
    extern __shared__ float4 smem4[];
    float2 *tw = reinterpret_cast<float2 *>(smem4);
    float2 *buf = tw + BM;                       // BM rows x PB: (k1, n1) at row 16 k1 + n1
    float *red = reinterpret_cast<float *>(buf + BM * PB);
    const int f = blockIdx.x / (BM / SLAB), cb = blockIdx.x % (BM / SLAB), j = a.j0 + f;
    if (MODE == B_PROX) {
        // this slab's Gamma (128 B) and sqrt f (64 B) of each frequency row, into
        // L2 while the column FFT runs
        const size_t gi = (size_t)j * BMM + (size_t)threadIdx.x * BM + cb * SLAB;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.gamma + gi));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.sqrtf_ + gi));
    }
    for (int k = threadIdx.x; k < BM; k += NTB) tw[k] = a.tw[k];
    // thread (hi, cl) owns column kc; hi is n1 in stage 1 and k1 in stage 2
    const int cl = threadIdx.x % SLAB, hi = threadIdx.x / SLAB, kc = cb * SLAB + cl;
    float2 x[BR];
    if (MODE == B_IFFT_IN) {
        // frequency rows k1 + 16 k2 of column kc (k1 = hi): the inverse stage 2 input
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = __ldg(a.in + (size_t)j * BMM + (size_t)(hi + BR * t) * BM + kc);
    } else {
        // column stage 1: DFT over n2 of the spatial rows n1 + 16 n2
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = a.T[((size_t)f * BM + hi + BR * t) * BM + kc];
        dft<BR, false>(x);
        __syncthreads();  // twiddles in place
#pragma unroll
        for (int s = 0; s < BR; ++s) buf[(hi + BR * s) * PB + cl] = cmul(x[s], tw[hi * s]);
        __syncthreads();
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = buf[(BR * hi + t) * PB + cl];
    }
    float part = 0.f;
    {   // column stage 2 (frequencies k1 + 16 k2), the elementwise step, inverse stage 2
        // this thread's Gamma and sqrt f (frequency rows hi + 16 t of column kc),
        // loaded before any Gamma store (the compiler may not move loads past those
        // stores)
        const size_t g0 = (size_t)j * BMM + (size_t)hi * BM + kc;
        float2 *gseg = a.gamma + g0;
        const float *fseg = a.sqrtf_ + g0;
        float2 gmv[MODE == B_PROX ? BR : 1];
        float sfv[MODE == B_PROX || MODE == B_LOSS ? BR : 1];
        if (MODE == B_PROX || MODE == B_LOSS) {
#pragma unroll
            for (int t = 0; t < BR; ++t) {
                // read once per iteration: streaming loads (evict first) keep the
                // intermediate T resident in L2
                sfv[t] = __ldcs(fseg + BR * t * BM);
                if (MODE == B_PROX) gmv[MODE == B_PROX ? t : 0] = __ldcs(gseg + BR * t * BM);
            }
        }
        if (MODE != B_IFFT_IN) dft<BR, false>(x);
        const float inv_m = 1.f / (float)BM;
#pragma unroll
        for (int t = 0; t < BR; ++t) {
            const int kr = hi + BR * t;
            if (MODE == B_PROX) {
                const float2 ax = cscale(x[t], inv_m);
                const float sf = sfv[t];
                const float2 gm = gmv[MODE == B_PROX ? t : 0];
                const float a2 = ax.x * ax.x + ax.y * ax.y;
                part += fabsf((a2 > 0.f ? a2 * rsqrtf(a2) : 0.f) - sf);
                const float2 y = cadd(gm, ax);
                const float2 z = stagm_prox(y, sf, a.pc);
                const float2 gn = csub(y, z);
                __stcs(gseg + BR * t * BM, gn);
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
                x[t] = cscale(x[t], inv_m * __ldg(a.mask + kr * BM + kc));
            } else if (MODE == B_FWD_OUT) {
                a.out[(size_t)j * BMM + kr * BM + kc] = cscale(x[t], inv_m);
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
    {   // inverse column stage 1 -> spatial rows n1 + 16 n2 (n1 = hi)
#pragma unroll
        for (int s = 0; s < BR; ++s) x[s] = cmulc(buf[(hi + BR * s) * PB + cl], tw[hi * s]);
        dft<BR, true>(x);
#pragma unroll
        for (int t = 0; t < BR; ++t) a.T[((size_t)f * BM + hi + BR * t) * BM + kc] = x[t];
    }
}

__global__ void __launch_bounds__(NTB) rows_inv256_kernel(PassC a, const float2 *twg)
{
    extern __shared__ float4 smem4[];
    float2 *tw = reinterpret_cast<float2 *>(smem4);
    float2 *buf = tw + BM;  // SLAB rows x PX: inverse stage-2 output (k1, n1) at 17 k1 + n1
    const int f = blockIdx.x / (BM / SLAB), rb = blockIdx.x % (BM / SLAB), j = a.j0 + f;
    for (int k = threadIdx.x; k < BM; k += NTB) tw[k] = twg[k];
    // thread (r, lo): inverse stage 2 at k1 = lo, inverse stage 1 at n1 = lo
    const int lo = threadIdx.x % BR, r = threadIdx.x / BR, row = rb * SLAB + r;
    float2 x[BR];
    {   // inverse row stage 2: DFT over k2 of the frequencies k1 + 16 k2
        const float2 *src = a.T + ((size_t)f * BM + row) * BM + lo;
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = src[BR * t];
        dft<BR, true>(x);
        float2 *rp = buf + r * PX + (BR + 1) * lo;
#pragma unroll
        for (int t = 0; t < BR; ++t) rp[t] = x[t];
    }
    __syncthreads();  // (and the twiddles)
    {   // the block has read its slab of T, which nothing reads again: drop its 256
        // L2 lines without writing them back (saves the DRAM write of dead data)
        const float2 *line = a.T + ((size_t)f * BM + rb * SLAB) * BM + (size_t)threadIdx.x * (128 / sizeof(float2));
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(line) : "memory");
    }
    {   // inverse row stage 1 -> spatial columns n1 + 16 n2
        const float2 *rp = buf + r * PX + lo;
#pragma unroll
        for (int s = 0; s < BR; ++s) x[s] = cmulc(rp[(BR + 1) * s], tw[lo * s]);
        dft<BR, true>(x);
    }
    // the output row `row`, columns lo + 16 t, with the mode tests and the
    // per-frame bases hoisted out of the loop
    const float sc = a.scale;
    if (a.slot) {  // nonblind gather slots: conj(w) o q_j at the pixel's rank
        const uint8_t *rk = a.rank + (size_t)j * BMM + row * BM + lo;
        const float2 *wc = a.wconj + row * BM + lo;
        float2 *sl = a.slot + a.frame_base[j] + (size_t)row * a.frame_pitch[j] + lo;
        const size_t stride = (size_t)a.slot_stride;
#pragma unroll
        for (int t = 0; t < BR; ++t)
            sl[__ldg(rk + BR * t) * stride + BR * t] = cmulc(cscale(x[t], sc), __ldg(wc + BR * t));
    } else {
        float2 *o = a.out + (size_t)j * BMM + row * BM + lo;
        if (a.wconj) {
            const float2 *wc = a.wconj + row * BM + lo;
#pragma unroll
            for (int t = 0; t < BR; ++t) o[BR * t] = cmulc(cscale(x[t], sc), __ldg(wc + BR * t));
        } else {
#pragma unroll
            for (int t = 0; t < BR; ++t) __stcs(o + BR * t, cscale(x[t], sc));
        }
    }
}

// ---------------------------------------------------------------- single-pass frame update
// One thread-block cluster of CL CTAs holds one 256 x 256 frame in its
// distributed shared memory, so the frame crosses HBM once per direction and
// no intermediate leaves the chip.  CTA c of the cluster owns rows
// [RPC c, RPC c + RPC) of the frame while the rows are transformed (buffer A)
// and column frequencies [CPC c, CPC c + CPC) while the columns are (buffer B).
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
    static constexpr int CPC = BM / CL;  // column frequencies per CTA in the column phase
    static constexpr int NT = BR * RPC;  // one 16-point DFT per thread and stage
    static constexpr int MINB = 768 / NT;
    static constexpr int PR = BR * (BR + 1) + 1;  // buffer A pitch (rows hold 16 groups of 17)
    static constexpr int PC = CPC + 2;   // buffer B pitch (spread banks)
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
    float2 *bufB = bufA + K::A_ELEMS;  // column frequencies CPC c ..: BM x PC
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
    // this CTA's Gamma and sqrt f columns of every frequency row, into L2 while
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
    // ---- rows, stage 2: DFTs over n1 -> frequencies s + 16 t; first exchange
    {
        const int r = tid % RPC, s = tid / RPC;
        float2 x[BR];
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = bufA[r * PR + BR * s + t];
        dft<BR, false>(x);
        if (tid == 0) tbar_expect(&bar[0], K::XBYTES);
        cluster_wait();  // the receivers' barriers are initialised
        // column frequency s + 16 t of row RPC c + r belongs to CTA (s + 16 t) / CPC
        const unsigned bufB_row = smem_addr(bufB + (RPC * c + r) * PC), bar0 = smem_addr(&bar[0]);
#pragma unroll
        for (int t = 0; t < BR; ++t) {
            const int kc = s + BR * t;
            const unsigned dst = (unsigned)(kc / CPC);
            st_async_v2(cluster_addr(bufB_row + (unsigned)(sizeof(float2) * (kc % CPC)), dst), x[t],
                        cluster_addr(bar0, dst));
        }
    }
    if (!tbar_wait(&bar[0])) *a.err = 1;  // every CTA's share of this CTA's columns has arrived
    // ---- columns, stage 1: DFTs over t at n1 of column frequency CPC c + col
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
    // updateM-1-multi) on frequency rows s + 16 t, inverse stage 2
    float part = 0.f;
    {
        const int col = tid % CPC, s = tid / CPC, kc = CPC * c + col;
        float2 x[BR];
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = bufB[(BR * s + t) * PC + col];
        float2 gmv[BR];
        float sfv[BR];
        const float2 *gp = a.gamma + fo + (size_t)s * BM + kc;
        const float *fp = a.sqrtf_ + fo + (size_t)s * BM + kc;
#pragma unroll
        for (int t = 0; t < BR; ++t) {
            sfv[t] = __ldg(fp + BR * t * BM);
            gmv[t] = gp[BR * t * BM];
        }
        dft<BR, false>(x);
        const float inv_m = 1.f / (float)BM;
        float2 *gw = a.gamma + fo + (size_t)s * BM + kc;
#pragma unroll
        for (int t = 0; t < BR; ++t) {
            const float2 ax = cscale(x[t], inv_m);
            const float sf = sfv[t];
            const float a2 = ax.x * ax.x + ax.y * ax.y;
            part += fabsf((a2 > 0.f ? a2 * rsqrtf(a2) : 0.f) - sf);
            const float2 y = cadd(gmv[t], ax);
            const float2 z = stagm_prox(y, sf, a.pc);
            const float2 gn = csub(y, z);
            gw[BR * t * BM] = gn;
            x[t] = csub(z, gn);
        }
        dft<BR, true>(x);
#pragma unroll
        for (int t = 0; t < BR; ++t) bufB[(BR * s + t) * PC + col] = x[t];
    }
    __syncthreads();
    // ---- columns, inverse stage 1 -> spatial rows n1 + 16 t; second exchange
    {
        const int col = tid % CPC, n1 = tid / CPC, kc = CPC * c + col;
        float2 x[BR];
#pragma unroll
        for (int s = 0; s < BR; ++s) x[s] = cmulc(bufB[(n1 + BR * s) * PC + col], tw[n1 * s]);
        dft<BR, true>(x);
        if (tid == 0) tbar_expect(&bar[1], K::XBYTES);
#pragma unroll
        for (int t = 0; t < BR; ++t) {
            const int R = n1 + BR * t;  // spatial row, owned by CTA R / RPC
            const unsigned dst = (unsigned)(R / RPC);
            st_async_v2(cluster_addr(smem_addr(bufA + (R % RPC) * PR + kc), dst), x[t],
                        cluster_addr(smem_addr(&bar[1]), dst));
        }
    }
    if (!tbar_wait(&bar[1])) *a.err = 1;  // this CTA's rows have arrived
    // ---- rows, inverse stage 2: DFTs over k2 of the frequencies s + 16 k2
    {
        const int r = tid % RPC, s = tid / RPC;
        float2 *rp = bufA + r * PR;
        float2 x[BR];
#pragma unroll
        for (int t = 0; t < BR; ++t) x[t] = rp[s + BR * t];
        dft<BR, true>(x);
        __syncthreads();  // every frequency has been read
#pragma unroll
        for (int t = 0; t < BR; ++t) rp[(BR + 1) * s + t] = x[t];  // (k1, n1) at 17 k1 + n1
    }
    __syncthreads();
    // ---- rows, inverse stage 1 -> spatial columns n1 + 16 t; q_j, or conj(w) q_j
    // into the gather slots (nonblind)
    {
        const int n1 = tid % BR, r = tid / BR, row = RPC * c + r;
        const float2 *rp = bufA + r * PR;
        float2 x[BR];
#pragma unroll
        for (int s = 0; s < BR; ++s) x[s] = cmulc(rp[(BR + 1) * s + n1], tw[n1 * s]);
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

constexpr size_t SMEM_A = sizeof(float2) * (BM + SLAB * PX);
constexpr size_t SMEM_B = sizeof(float2) * (BM + BM * PB) + sizeof(float) * (NTB / 32);

// One pass-A / pass-B / pass-C sequence over frames [j0, j0 + J) in waves.
struct Pipeline {
    bool do_a, do_c;
    PassA A;
    PassB B;
    PassC C;
};

// Waves go round-robin to the plan's chains (t_waves) -- the caller's stream
// and the plan's wave streams, each chain with its own T buffer -- so that the
// blocks of one chain's pass fill the SMs that another chain's pass leaves idle
// at its tail, and the DRAM-bound column pass of one wave runs beside the
// L2-bound row passes of others.  The chains fork from and join back into the
// caller's stream (inside a graph capture these become graph edges).
int run_waves(const ptycho_plan_s *p, Pipeline P, int J, int waves_frames, cudaStream_t s)
{
    const int slabs = BM / SLAB;
    const int nch = std::max(1, std::min(p->t_waves, (J + waves_frames - 1) / waves_frames));
    cudaStream_t st[MAX_WAVE_CHAINS];
    float2 *T[MAX_WAVE_CHAINS];
    for (int c = 0; c < nch; ++c) {
        st[c] = c ? p->wave_stream[c] : s;
        T[c] = p->d_T + (size_t)c * p->wave_frames * BMM;
    }
    if (nch > 1) {
        OD2P_CUDA(cudaEventRecord(p->wave_ev[0], s));
        for (int c = 1; c < nch; ++c) OD2P_CUDA(cudaStreamWaitEvent(st[c], p->wave_ev[0], 0));
    }
    cudaError_t e = cudaSuccess;
    for (int w0 = 0, wi = 0; w0 < J && e == cudaSuccess; w0 += waves_frames, ++wi) {
        const int nf = std::min(waves_frames, J - w0), ch = wi % nch;
        const cudaStream_t sw = st[ch];
        if (P.do_a) {
            PassA a = P.A;
            a.j0 = w0;
            a.nf = nf;
            a.T = T[ch];
            rows_fwd256_kernel<<<nf * slabs, NTB, SMEM_A, sw>>>(a);
            e = cudaGetLastError();
        }
        PassB b = P.B;
        b.j0 = w0;
        b.nf = nf;
        b.part_off = w0 * slabs;
        b.T = T[ch];
        if (e == cudaSuccess) {
            switch (b.mode) {
            case B_PROX: cols256_kernel<B_PROX><<<nf * slabs, NTB, SMEM_B, sw>>>(b); break;
            case B_FWD_OUT: cols256_kernel<B_FWD_OUT><<<nf * slabs, NTB, SMEM_B, sw>>>(b); break;
            case B_LOSS: cols256_kernel<B_LOSS><<<nf * slabs, NTB, SMEM_B, sw>>>(b); break;
            case B_MASK: cols256_kernel<B_MASK><<<nf * slabs, NTB, SMEM_B, sw>>>(b); break;
            default: cols256_kernel<B_IFFT_IN><<<nf * slabs, NTB, SMEM_B, sw>>>(b); break;
            }
            e = cudaGetLastError();
        }
        if (P.do_c && e == cudaSuccess) {
            PassC c = P.C;
            c.j0 = w0;
            c.nf = nf;
            c.T = T[ch];
            rows_inv256_kernel<<<nf * slabs, NTB, SMEM_A, sw>>>(c, P.B.tw);
            e = cudaGetLastError();
        }
    }
    for (int c = 1; c < nch; ++c) {  // join even after a failed launch, so that a capture can end
        const cudaError_t e1 = cudaEventRecord(p->wave_ev[c], st[c]);
        const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(s, p->wave_ev[c], 0) : e1;
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) return cuda_fail(e, "m = 256 frame passes");
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
        const float v = sqrtf(fmaxf(__ldg(f + (size_t)j * BMM + k), 0.f));
        sqrtf_[(size_t)j * BMM + k] = v;  // natural order
        acc += v;
    }
    const float tot = block_sum_fixed(acc, red);
    if (threadIdx.x == 0) part[j] = tot;
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
    return run_waves(p, P, p->J, p->wave_frames, s);
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
    return run_waves(p, P, p->J, p->wave_frames, s);
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
    return run_waves(p, P, p->J, p->wave_frames, s);
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
    return run_waves(p, P, p->J, p->wave_frames, s);
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
    return run_waves(p, P, p->J, p->wave_frames, s);
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
    return run_waves(p, P, 1, 1, s);
}

int ingest_256(ptycho_plan_s *p, const float *f, float *part, cudaStream_t s)
{
    ingest256_kernel<<<p->J, 256, 0, s>>>(p->J, f, p->d_sqrtf, part);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

// m = 256 keeps Gamma in natural order: getting or setting it is a copy
int permute_256(const ptycho_plan_s *p, const float2 *src, float2 *dst, bool, cudaStream_t s)
{
    if (src != dst)
        OD2P_CUDA(cudaMemcpyAsync(dst, src, sizeof(float2) * (size_t)p->J * BMM, cudaMemcpyDeviceToDevice, s));
    return PTYCHO_OK;
}

}  // namespace od2p
