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
        // Gamma and sqrt f of the thread's column segment, loaded before any
        // Gamma store (the compiler may not move loads past those stores)
        float2 gmv[MODE == B_PROX ? BR : 1];
        float sfv[MODE == B_PROX || MODE == B_LOSS ? BR : 1];
        if (MODE == B_PROX || MODE == B_LOSS) {
#pragma unroll
            for (int t = 0; t < BR; ++t) {
                const size_t gi = (size_t)j * BMM + (size_t)(BR * hi + t) * BM + pc;
                sfv[t] = __ldg(a.sqrtf_ + gi);
                if (MODE == B_PROX) gmv[MODE == B_PROX ? t : 0] = a.gamma[gi];
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
                a.gamma[gi] = gn;
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
    for (int r = 0; r < SLAB; ++r) {
        const int row = rb * SLAB + r;
        float2 v = cscale(buf[r * PA + c], a.scale);
        if (a.wconj) v = cmulc(v, __ldg(a.wconj + row * BM + c));
        if (a.slot)
            a.slot[(size_t)__ldg(a.rank + (size_t)j * BMM + row * BM + c) * a.slot_stride + a.frame_base[j] +
                   row * a.frame_pitch[j] + c] = v;
        else
            a.out[(size_t)j * BMM + row * BM + c] = v;
    }
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

int frame_update_256(ptycho_plan_s *p, cudaStream_t s)
{
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

int loss_256(ptycho_plan_s *p, const float2 *u, const float2 *w, cudaStream_t s)
{
    Pipeline P = base_pipeline(p);
    P.do_a = P.do_c = true;
    P.A.frame_base = p->d_img_base;
    P.A.frame_pitch = p->d_img_pitch;
    P.A.u = u;
    P.A.w = w;
    P.B.mode = B_LOSS;
    P.B.part = p->d_loss_part;
    P.C.out = p->d_q;
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
