// Image-space kernels of the OD2P library for sm_103a: the deterministic
// gather-form overlap-add fused with the consensus v, u and Lambda updates
// (Algorithm 2 Steps 1 (v), 3 and 4; Algorithm 3 Steps 4 and 5), the image
// gather of the adjoint, the fixed-order probe reductions of the blind
// W-update (Algorithm 3 Step 3) and of grad_w, and small helpers.
//
// Determinism: every pixel sums the frames covering it in ascending j (the
// per-tile frame lists are ascending), every reduction runs in a fixed order,
// and no kernel uses atomics, so repeated runs are bitwise identical.
#include "od2p_internal.h"

namespace od2p {
namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// conj(a) * b
__device__ __forceinline__ float2 cconjmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

// Fixed-order sum of n values v[i * stride + offset] by one warp: lane l adds
// the contiguous run [l*per, (l+1)*per) in order, then a fixed shuffle tree.
// Every lane returns the total.  Deterministic for a given n.
__device__ __forceinline__ double warp_sum_runs(int n, const float *v, int stride, int offset)
{
    const int lane = threadIdx.x & 31, per = (n + 31) / 32;
    double t = 0.0;
    for (int i = lane * per; i < min(n, (lane + 1) * per); ++i) t += v[(size_t)i * stride + offset];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    return __shfl_sync(0xffffffffu, t, 0);
}

__device__ __forceinline__ void block_sum2_fixed(float &a, float &b, float *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[2 * warp] = a;
        red[2 * warp + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float ta = 0.f, tb = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            ta += red[2 * i];
            tb += red[2 * i + 1];
        }
        a = ta;
        b = tb;
    }
}

// ---------------------------------------------------------------- K2: subdomain update

// One block per TILE_H x TILE_W tile; lane = column, warp w owns rows
// [w * TILE_ROWS, (w + 1) * TILE_ROWS) of it.  The tile's frame list (ascending
// j) is staged in shared memory; per entry the row test is warp-uniform, the
// column test per lane, and the entry's TILE_ROWS loads are independent.
// Each pixel adds its frames in list order.  Only the neighbours whose
// rectangles meet the tile are visited (interior tiles have none).
constexpr int LIST_SMEM = 160;
constexpr int NBR_SMEM = 16;

// One plan: block b updates tile b with the arguments `single`.  Batches:
// block b updates tile items[b].y of the plan whose arguments are
// tab[2 items[b].x + parity].
#ifndef OD2P_K2_U
#define OD2P_K2_U 4
#endif
#ifndef OD2P_K2_MINB
#define OD2P_K2_MINB 4
#endif
#ifndef OD2P_K2B_U
#define OD2P_K2B_U 1
#endif
#ifndef OD2P_K2B_MINB
#define OD2P_K2B_MINB 4
#endif
#ifndef OD2P_PROBE_U
#define OD2P_PROBE_U 4
#endif
template <bool BLIND, bool BATCHED>
__global__ void __launch_bounds__(GATHER_THREADS, BLIND ? OD2P_K2B_MINB : OD2P_K2_MINB)
    subdomain_update_kernel(const SubArgs single, const SubArgs *__restrict__ tab, const int2 *__restrict__ items,
                            int parity)
{
    __shared__ float red[2 * (GATHER_THREADS / 32)];
    __shared__ ListEntry lst[BLIND ? LIST_SMEM : 1];
    __shared__ NbrInfo nbs[NBR_SMEM];
    __shared__ SubArgs sa;
    const int2 it = BATCHED ? items[blockIdx.x] : make_int2(0, (int)blockIdx.x);
    if (BATCHED) {
        if (threadIdx.x == 0) sa = tab[2 * it.x + parity];
        __syncthreads();
    }
    const SubArgs &a = BATCHED ? sa : single;
    const int tix = it.y;
    const TileInfo ti = a.tinfo[tix];
    const int lane = threadIdx.x & 31, ty0 = (threadIdx.x >> 5) * TILE_ROWS;
    const bool col_ok = lane < ti.ncols;
    const int nrows = min(TILE_ROWS, ti.nrows - ty0);  // rows of this thread inside Omega_d (may be <= 0)
    const bool active = col_ok && nrows > 0;
    const int C = ti.C0 + lane, R0 = ti.R0 + ty0;
    const int M = a.M, MM = M * M;
    // u index of each of the thread's rows (the last valid row repeated)
    int ui[TILE_ROWS];
#pragma unroll
    for (int r = 0; r < TILE_ROWS; ++r) ui[r] = ti.u0 + (ty0 + max(0, min(r, nrows - 1))) * ti.pitch + lane;
    int nk_r[TILE_ROWS];
#pragma unroll
    for (int r = 0; r < TILE_ROWS; ++r) nk_r[r] = (!BLIND && active && r < nrows) ? (int)__ldg(a.cnt + ui[r]) : 0;
    if (BLIND)
        for (int i = threadIdx.x; i < min(ti.nk, LIST_SMEM); i += GATHER_THREADS) lst[i] = a.tlist[ti.k0 + i];
    for (int i = threadIdx.x; i < min(ti.nnb, NBR_SMEM); i += GATHER_THREADS) nbs[i] = a.tnbr[ti.n0 + i];
    __syncthreads();
    // A_d^*(z - Gamma) at each pixel, frames in ascending j.  Nonblind: the
    // slots already carry conj(w) and sum_j S_j^T |w|^2 is precomputed.  Blind:
    // weight with W_d^{n+1} here and sum |W_d|^2 on the way.
    float2 acc[TILE_ROWS];
    float nrm[TILE_ROWS];
#pragma unroll
    for (int r = 0; r < TILE_ROWS; ++r) {
        acc[r] = make_float2(0.f, 0.f);
        nrm[r] = 0.f;
    }
    const float2 *w = BLIND ? a.Wd + ti.reg * a.wd_stride : nullptr;
    if (!BLIND) {
        // nonblind: the pixel's frames sit in slots 0 .. cnt-1 in ascending j;
        // U slots x TILE_ROWS rows of coalesced, independent loads per step; a
        // row past its count loads slot 0 and discards it
        if (active) {
            int kmax = 0;
#pragma unroll
            for (int r = 0; r < TILE_ROWS; ++r) kmax = max(kmax, nk_r[r]);
            constexpr int U = OD2P_K2_U;
            for (int k = 0; k < kmax; k += U) {
                float2 v[U][TILE_ROWS];
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int r = 0; r < TILE_ROWS; ++r) {
                        const unsigned kk = k + u < nk_r[r] ? (unsigned)(k + u) : 0u;
                        // 32-bit index: the plan checks slot_k * u_len < 2^32
                        v[u][r] = __ldg(a.slot + (kk * (unsigned)a.slot_stride + (unsigned)ui[r]));
                    }
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int r = 0; r < TILE_ROWS; ++r)
                        if (k + u < nk_r[r]) acc[r] = cadd(acc[r], v[u][r]);
            }
        }
    } else if (active) {
        // blind: walk the tile's frame list and weight with W_d^{n+1};
        // U entries x TILE_ROWS rows of loads per step, branch-free: a lane whose
        // pixel a frame does not cover loads element 0 and discards it.
        constexpr int U = OD2P_K2B_U;
        const int nk = ti.nk;
        for (int k = 0; k < nk; k += U) {
            float2 qv[U][TILE_ROWS], wv[U][TILE_ROWS];
            unsigned hits = 0u;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool valid = k + u < nk;
                const ListEntry e = valid ? (k + u < LIST_SMEM ? lst[k + u] : a.tlist[ti.k0 + k + u]) : ListEntry{0, M, M, 0};
                const int dr0 = e.dr + ty0, dc = e.dc + lane;
                const bool cok = (unsigned)dc < (unsigned)M;
#pragma unroll
                for (int r = 0; r < TILE_ROWS; ++r) {
                    const int dr = dr0 + r;
                    const bool hit = cok && r < nrows && (unsigned)dr < (unsigned)M;
                    const int o = hit ? dr * M + dc : 0;
                    qv[u][r] = __ldcs(a.q + (hit ? e.j * MM + o : 0));  // read once: evict first
                    if (w) wv[u][r] = __ldg(w + o);
                    hits |= (hit ? 1u : 0u) << (u * TILE_ROWS + r);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int r = 0; r < TILE_ROWS; ++r)
                    if (hits & (1u << (u * TILE_ROWS + r))) {
                        if (w) {
                            acc[r] = cadd(acc[r], cconjmul(wv[u][r], qv[u][r]));
                            nrm[r] += cabs2(wv[u][r]);
                        } else {
                            acc[r] = cadd(acc[r], qv[u][r]);
                        }
                    }
        }
    }
    float dn = 0.f, nn = 0.f;
    if (active) {
        float2 u_old[TILE_ROWS], num[TILE_ROWS], u_new[TILE_ROWS];
        float den[TILE_ROWS];
#pragma unroll
        for (int r = 0; r < TILE_ROWS; ++r) {
            u_old[r] = a.u_cur[ui[r]];
            num[r] = cscale(acc[r], a.eta);
            den[r] = a.eta * (BLIND ? nrm[r] : __ldg(a.nrm + ui[r]));
        }
        const int nnb = ti.nnb, n0 = ti.n0, rend = ti.rend;
        // consensus v_{d,e} (eq. updateV-multi) and the r-terms of the u-update:
        // one neighbour at a time, the loads of all rows together
        for (int i = 0; i < nnb; ++i) {
            const NbrInfo nb = i < NBR_SMEM ? nbs[i] : a.tnbr[n0 + i];
            if (C < nb.c0 || C >= nb.c1 || R0 + nrows <= nb.r0 || R0 >= nb.r1) continue;
            float2 ue[TILE_ROWS], lde[TILE_ROWS], led[TILE_ROWS];
#pragma unroll
            for (int r = 0; r < TILE_ROWS; ++r) {
                // clamped into Omega_d n Omega_e: rows outside are loaded but discarded
                const int R = min(max(R0 + r, nb.r0), min(nb.r1, rend) - 1);
                const int li = (R - nb.p_r0) * nb.p_pitch + (C - nb.p_c0);
                ue[r] = a.u_cur[nb.u_base + (R - nb.r0) * nb.u_pitch + (C - nb.c0)];
                lde[r] = a.lam_cur[nb.lam_de + li];
                led[r] = a.lam_cur[nb.lam_ed + li];
            }
#pragma unroll
            for (int r = 0; r < TILE_ROWS; ++r) {
                if (r >= nrows || R0 + r < nb.r0 || R0 + r >= nb.r1) continue;
                // same operand order on both sides of the pair -> bitwise equal v
                const float2 v = nb.d_first ? cscale(cadd(cadd(u_old[r], ue[r]), cadd(lde[r], led[r])), 0.5f)
                                            : cscale(cadd(cadd(ue[r], u_old[r]), cadd(led[r], lde[r])), 0.5f);
                num[r] = cadd(num[r], cscale(csub(v, lde[r]), a.r));
                den[r] += a.r;
            }
        }
#pragma unroll
        for (int r = 0; r < TILE_ROWS; ++r) {
            if (BLIND) {
                num[r] = cadd(num[r], cscale(u_old[r], a.gamma));
                den[r] += a.gamma;
            }
            // eq. Alg1-solver-u; a pixel with no illumination and no overlap keeps its value
            u_new[r] = den[r] > 0.f ? make_float2(num[r].x / den[r], num[r].y / den[r]) : u_old[r];
            if (r < nrows) {
                a.u_next[ui[r]] = u_new[r];
                dn += cabs2(csub(u_new[r], u_old[r]));
                nn += cabs2(u_new[r]);
            }
        }
        // eq. updateM-2-multi: Lambda_{d,e} += pi u_d^{n+1} - v
        for (int i = 0; i < nnb; ++i) {
            const NbrInfo nb = i < NBR_SMEM ? nbs[i] : a.tnbr[n0 + i];
            if (C < nb.c0 || C >= nb.c1 || R0 + nrows <= nb.r0 || R0 >= nb.r1) continue;
            float2 ue[TILE_ROWS], lde[TILE_ROWS], led[TILE_ROWS];
            int li[TILE_ROWS];
#pragma unroll
            for (int r = 0; r < TILE_ROWS; ++r) {
                const int R = min(max(R0 + r, nb.r0), min(nb.r1, rend) - 1);
                li[r] = (R - nb.p_r0) * nb.p_pitch + (C - nb.p_c0);
                ue[r] = a.u_cur[nb.u_base + (R - nb.r0) * nb.u_pitch + (C - nb.c0)];
                lde[r] = a.lam_cur[nb.lam_de + li[r]];
                led[r] = a.lam_cur[nb.lam_ed + li[r]];
            }
#pragma unroll
            for (int r = 0; r < TILE_ROWS; ++r) {
                if (r >= nrows || R0 + r < nb.r0 || R0 + r >= nb.r1) continue;
                const float2 v = nb.d_first ? cscale(cadd(cadd(u_old[r], ue[r]), cadd(lde[r], led[r])), 0.5f)
                                            : cscale(cadd(cadd(ue[r], u_old[r]), cadd(led[r], lde[r])), 0.5f);
                a.lam_next[nb.lam_de + li[r]] = csub(cadd(lde[r], u_new[r]), v);
            }
        }
    }
    block_sum2_fixed(dn, nn, red);
    if (threadIdx.x == 0) {
        a.re_part[2 * tix] = dn;
        a.re_part[2 * tix + 1] = nn;
    }
}

// ---------------------------------------------------------------- image gather
// out(p) = sum_{j covering p, ascending} (w ? conj(w(p - o_j)) : 1) * h_j(p - o_j)
__global__ void __launch_bounds__(GATHER_THREADS) image_gather_kernel(
    int M, int H, int W, const Tile *tiles, const int32_t *tptr, const ListEntry *tlist,
    const float2 *h, const float2 *w, float2 *out)
{
    const Tile tile = tiles[blockIdx.x];
    const int lane = threadIdx.x & 31, ty0 = (threadIdx.x >> 5) * TILE_ROWS;
    const int C = tile.c0 + lane, R0 = tile.r0 + ty0;
    const int nrows = min(TILE_ROWS, H - R0);
    if (C >= W || nrows <= 0) return;
    const int MM = M * M;
    float2 acc[TILE_ROWS];
#pragma unroll
    for (int r = 0; r < TILE_ROWS; ++r) acc[r] = make_float2(0.f, 0.f);
    // two list entries per step, branch-free: a lane whose pixel a frame does not
    // cover loads element 0 and discards it (sums stay in ascending j)
    constexpr int U = 2;
    const int k0 = tptr[blockIdx.x], k1 = tptr[blockIdx.x + 1];
    for (int k = k0; k < k1; k += U) {
        float2 hv[U][TILE_ROWS], wv[U][TILE_ROWS];
        unsigned hits = 0u;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const ListEntry e = k + u < k1 ? tlist[k + u] : ListEntry{0, M, M, 0};
            const int dr0 = e.dr + ty0, dc = e.dc + lane;
            const bool cok = (unsigned)dc < (unsigned)M;
#pragma unroll
            for (int r = 0; r < TILE_ROWS; ++r) {
                const int dr = dr0 + r;
                const bool hit = cok && r < nrows && (unsigned)dr < (unsigned)M;
                const int o = hit ? dr * M + dc : 0;
                hv[u][r] = __ldg(h + (hit ? (size_t)e.j * MM + o : 0));
                if (w) wv[u][r] = __ldg(w + o);
                hits |= (hit ? 1u : 0u) << (u * TILE_ROWS + r);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int r = 0; r < TILE_ROWS; ++r)
                if (hits & (1u << (u * TILE_ROWS + r)))
                    acc[r] = cadd(acc[r], w ? cconjmul(wv[u][r], hv[u][r]) : hv[u][r]);
    }
#pragma unroll
    for (int r = 0; r < TILE_ROWS; ++r)
        if (r < nrows) out[(size_t)(R0 + r) * W + C] = acc[r];
}

// ---------------------------------------------------------------- penalties and consensus
// x <- s x for n complex values (rescaling of a scaled multiplier).
__global__ void scale_kernel(int64_t n, float2 *x, float s)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        x[e] = cscale(x[e], s);
}

constexpr int RC_BLOCKS = 64;  // blocks per ordered pair / over u in the consensus residual

// part[k * RC_BLOCKS + b] = sum over block b's share (element-strided, fixed
// order) of |u_d - u_e|^2 on ordered pair k's overlap; part[P * RC_BLOCKS + b]
// likewise of |u|^2 over all subdomain pixels.
// pair_shift (null without periodic boundaries): u_e is read at (R - s_r H, C - s_c W)
__global__ void __launch_bounds__(256) consensus_partial_kernel(int P, const int32_t *pair, const int32_t *pair_rect,
                                                                const int32_t *pair_shift, int H, int W,
                                                                const int32_t *rect, const int64_t *u_off,
                                                                int64_t u_len, const float2 *u, float *part)
{
    __shared__ float red[2 * (256 / 32)];
    const int k = blockIdx.y;
    float acc = 0.f, dummy = 0.f;
    if (k < P) {
        const int d = pair[2 * k], e = pair[2 * k + 1];
        const int sR = pair_shift ? pair_shift[2 * k] * H : 0, sC = pair_shift ? pair_shift[2 * k + 1] * W : 0;
        const int32_t *pr = pair_rect + 4 * k, *Rd = rect + 4 * d, *Re = rect + 4 * e;
        const int w = pr[3] - pr[1];
        const int64_t n = (int64_t)(pr[2] - pr[0]) * w;
        for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += RC_BLOCKS * 256) {
            const int R = pr[0] + (int)(i / w), C = pr[1] + (int)(i % w);
            const float2 a = u[u_off[d] + (int64_t)(R - Rd[0]) * (Rd[3] - Rd[1]) + (C - Rd[1])];
            const float2 b = u[u_off[e] + (int64_t)(R - sR - Re[0]) * (Re[3] - Re[1]) + (C - sC - Re[1])];
            acc += cabs2(csub(a, b));
        }
    } else {
        for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < u_len; i += RC_BLOCKS * 256) acc += cabs2(u[i]);
    }
    block_sum2_fixed(acc, dummy, red);
    if (threadIdx.x == 0) part[(size_t)k * RC_BLOCKS + blockIdx.x] = acc;
}

// out = sqrt(sum over the pairs' parts / sum of the |u|^2 parts), fixed order.
// One warp.
__global__ void consensus_final_kernel(int P, const float *part, double *out)
{
    const double num = warp_sum_runs(P * RC_BLOCKS, part, 1, 0);
    const double den = warp_sum_runs(RC_BLOCKS, part + (size_t)P * RC_BLOCKS, 1, 0);
    if (threadIdx.x == 0) *out = den > 0.0 ? sqrt(num / den) : 0.0;
}

// ---------------------------------------------------------------- probe reductions
// Level 1: per chunk of PROBE_CHUNK frames of one group, for every probe pixel k:
//   part[c][k] = sum_{j in chunk, ascending} conj(u(o_j + k)) h_j(k), part_n = sum |u(o_j + k)|^2.
struct ProbeArgs {
    int32_t M;
    const int4 *chunks;          // (group, begin, end, -) into group_frames
    const int32_t *group_frames; // frame ids, ascending within each group
    const int32_t *frame_base;   // index of the window origin in u
    const int32_t *frame_pitch;  // per-frame pitch, or null for `pitch`
    int32_t pitch;
    const float2 *u, *h;
    float2 *part;
    float *part_n;
};

__global__ void probe_partial_kernel(ProbeArgs a)
{
    const int MM = a.M * a.M;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= MM) return;
    const int4 ch = a.chunks[blockIdx.y];
    const int kr = k / a.M, kc = k % a.M;
    float2 acc = make_float2(0.f, 0.f);
    float nn = 0.f;
    // U frames' loads in flight per step, accumulated in ascending order
    constexpr int U = OD2P_PROBE_U;
    for (int t0 = ch.y; t0 < ch.z; t0 += U) {
        float2 uv[U], hv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = min(t0 + u, ch.z - 1);
            const int j = a.group_frames[t];
            const int pitch = a.frame_pitch ? a.frame_pitch[j] : a.pitch;
            uv[u] = __ldg(a.u + a.frame_base[j] + (size_t)kr * pitch + kc);
            hv[u] = __ldcs(a.h + (size_t)j * MM + k);  // read once per pass: evict first
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (t0 + u < ch.z) {
                acc = cadd(acc, cconjmul(uv[u], hv[u]));
                nn += cabs2(uv[u]);
            }
    }
    a.part[(size_t)blockIdx.y * MM + k] = acc;
    a.part_n[(size_t)blockIdx.y * MM + k] = nn;
}

// Level 2 (blind, eqs. blind_W and admm_Delta): per subdomain d and pixel k,
// N = sum of its chunks in order, Dn likewise;
// W_d = (eta N + mu (w^{n+1} - Delta_d)) / (eta Dn + mu); Delta_d += W_d - w^{n+1}.
__global__ void probe_finalize_blind_kernel(int M, int D, const int32_t *group_chunk_ptr,
                                            const float2 *part, const float *part_n,
                                            const float2 *wnew, float2 *Wd, float2 *Delta,
                                            float eta, float mu)
{
    const int MM = M * M;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    if (k >= MM || d >= D) return;
    float2 N = make_float2(0.f, 0.f);
    float Dn = 0.f;
    for (int c = group_chunk_ptr[d]; c < group_chunk_ptr[d + 1]; ++c) {
        N = cadd(N, part[(size_t)c * MM + k]);
        Dn += part_n[(size_t)c * MM + k];
    }
    const float2 wn = wnew[k];
    const float2 dl = Delta[(size_t)d * MM + k];
    const float den = eta * Dn + mu;
    const float2 num = cadd(cscale(N, eta), cscale(csub(wn, dl), mu));
    const float2 Wn = make_float2(num.x / den, num.y / den);
    Wd[(size_t)d * MM + k] = Wn;
    Delta[(size_t)d * MM + k] = cadd(dl, csub(Wn, wn));
}

__global__ void probe_finalize_sum_kernel(int M, int n_chunks, const float2 *part, float2 *out)
{
    const int MM = M * M;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= MM) return;
    float2 N = make_float2(0.f, 0.f);
    for (int c = 0; c < n_chunks; ++c) N = cadd(N, part[(size_t)c * MM + k]);
    out[k] = N;
}

// ---------------------------------------------------------------- scalars
// Fixed-order sum of n values with one NT-thread block: thread t adds the
// contiguous run [t*per, (t+1)*per) in order, then a fixed shuffle tree and
// the NT/32 warp sums in order.  Deterministic for a given n and NT.
template <int NT>
__device__ double block_sum_runs(int n, const float *v, int stride, int offset, double *red)
{
    const int per = (n + NT - 1) / NT;
    double t = 0.0;
    for (int i = threadIdx.x * per; i < min(n, (threadIdx.x + 1) * per); ++i) t += v[(size_t)i * stride + offset];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < NT / 32; ++i) s += red[i];
    return s;
}

// metrics[0] = sum rf_part / sum sqrt f (RF); metrics[1] = max over subdomains of
// sqrt(sum dn / sum nn) over the subdomain's tiles (RE).  One block of 1024
// threads: RF by the block, then warp k takes subdomains k, k + 32, ...
// (fixed-order sums each).
__global__ void __launch_bounds__(1024) metrics_kernel(int n_rf, const float *rf_part, int D,
                                                       const int32_t *reg_tile_ptr, const float *re_part,
                                                       double *metrics)
{
    __shared__ double red[32];
    __shared__ double re_w[32];
    const double rf = block_sum_runs<1024>(n_rf, rf_part, 1, 0, red);
    const int warp = threadIdx.x >> 5;
    double re = 0.0;
    for (int d = warp; d < D; d += 32) {
        const int t0 = reg_tile_ptr[d], nt = reg_tile_ptr[d + 1] - t0;
        const double dn = warp_sum_runs(nt, re_part + 2 * (size_t)t0, 2, 0);
        const double nn = warp_sum_runs(nt, re_part + 2 * (size_t)t0, 2, 1);
        const double v = nn > 0.0 ? sqrt(dn / nn) : 0.0;
        re = v > re ? v : re;
    }
    if ((threadIdx.x & 31) == 0) re_w[warp] = re;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < 32; ++k) re = re_w[k] > re ? re_w[k] : re;
        metrics[0] = metrics[2] > 0.0 ? rf / metrics[2] : 0.0;
        metrics[1] = re;
    }
}

// ---- iterate-until: the stopping test of section 4 evaluated on the device
// st[0] iterations done, st[1] the cap, st[2] the RF tolerance (float bits),
// st[3] the last RF (float bits).
__global__ void until_init_kernel(int32_t *st, int32_t max_iter, float tol)
{
    st[0] = 0;
    st[1] = max_iter;
    st[2] = __float_as_int(tol);
    st[3] = __float_as_int(0.f);
}

// Conditional-node self check: set a handle, and mark from the body it guards.
__global__ void cond_set_kernel(cudaGraphConditionalHandle h, unsigned value)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h, value);
}
__global__ void cond_mark_kernel(int32_t *flag)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *flag = 1;
}

// After each iteration of the graph's loop: RF of that iteration (the same
// fixed-order sum as od2p_metrics), then continue while (float) RF > tol and
// fewer than the cap; the decision sets the loop's condition and, inside the
// loop body, the condition of its second iteration.
__global__ void __launch_bounds__(1024) until_check_kernel(int n_rf, const float *rf_part, const double *metrics,
                                                            int32_t *st, cudaGraphConditionalHandle h_loop,
                                                            cudaGraphConditionalHandle h_second, int set_second)
{
    __shared__ double red[32];
    const double rf = block_sum_runs<1024>(n_rf, rf_part, 1, 0, red);
    if (threadIdx.x != 0) return;
    const float v = (float)(metrics[2] > 0.0 ? rf / metrics[2] : 0.0);
    const int n = st[0] + 1;
    st[0] = n;
    st[3] = __float_as_int(v);
    const unsigned go = (v > __int_as_float(st[2]) && n < st[1]) ? 1u : 0u;
    cudaGraphSetConditional(h_loop, go);
    if (set_second) cudaGraphSetConditional(h_second, go);
}

__global__ void __launch_bounds__(256) sum_kernel(int n, const float *part, double *dst)
{
    __shared__ double red[8];
    const double t = block_sum_runs<256>(n, part, 1, 0, red);
    if (threadIdx.x == 0) *dst = t;
}

__global__ void __launch_bounds__(256) loss_sum_kernel(int n, const float *part, float *loss)
{
    __shared__ double red[8];
    const double t = block_sum_runs<256>(n, part, 1, 0, red);
    if (threadIdx.x == 0) *loss = (float)t;
}

// sum_j S_j^T |w|^2 over each subdomain's frames (ascending j), per subdomain
// pixel: the diagonal of A_d^* A_d (eq. AtA) for the known probe.
__global__ void __launch_bounds__(GATHER_THREADS) illumination_kernel(int M, const int32_t *rect,
                                                                      const int64_t *u_off, const Tile *tiles,
                                                                      const int32_t *tptr, const ListEntry *tlist,
                                                                      const float2 *w, float *nrm)
{
    const Tile tile = tiles[blockIdx.x];
    const int32_t *rc = rect + 4 * tile.reg;
    const int hd = rc[2] - rc[0], wd = rc[3] - rc[1];
    const int lane = threadIdx.x & 31, ty0 = (threadIdx.x >> 5) * TILE_ROWS;
    const int lc = tile.c0 + lane;
    if (lc >= wd) return;
    for (int r = 0; r < TILE_ROWS; ++r) {
        const int lr = tile.r0 + ty0 + r;
        if (lr >= hd) break;
        float acc = 0.f;
        for (int k = tptr[blockIdx.x]; k < tptr[blockIdx.x + 1]; ++k) {
            const ListEntry e = tlist[k];
            const int dr = e.dr + ty0 + r, dc = e.dc + lane;
            if ((unsigned)dr < (unsigned)M && (unsigned)dc < (unsigned)M) acc += cabs2(__ldg(w + dr * M + dc));
        }
        nrm[u_off[tile.reg] + (int64_t)lr * wd + lc] = acc;
    }
}

// Offset of frame pixel (row, col) in a frame's slot ranks.  m <= 128: task
// order -- the frame update's column task (n1 = row % R2, col) holds the R1
// ranks of rows n1, n1 + R2, ... contiguously, so that one thread loads them
// with one vector load; m = 256 (R1 = 0): natural row-major order.
__device__ __forceinline__ int rank_offset(int M, int R1, int R2, int row, int col)
{
    return R1 ? ((row % R2) * M + col) * R1 + row / R2 : row * M + col;
}

// Gather slots of a nonblind plan: the rank of every frame pixel among the
// frames of its subdomain that cover the same subdomain pixel (ascending j: the
// tile lists are ascending), and the number of covering frames per pixel.  Each
// frame pixel lies in exactly one tile of its own subdomain, so every rank is
// written once.  setup[0] is set when a pixel has more than 255 frames, setup[1]
// receives the largest count (atomicMax: an integer maximum, order-free).
__global__ void __launch_bounds__(GATHER_THREADS) slot_rank_kernel(int M, int R1, int R2, const TileInfo *tinfo,
                                                                   const ListEntry *tlist, uint8_t *rank,
                                                                   uint8_t *cnt, int32_t *setup)
{
    const TileInfo ti = tinfo[blockIdx.x];
    const int lane = threadIdx.x & 31, ty0 = (threadIdx.x >> 5) * TILE_ROWS;
    if (lane >= ti.ncols) return;
    const int MM = M * M;
    int most = 0;
    for (int r = 0; r < TILE_ROWS && ty0 + r < ti.nrows; ++r) {
        int n = 0;
        for (int k = 0; k < ti.nk; ++k) {
            const ListEntry e = tlist[ti.k0 + k];
            const int dr = e.dr + ty0 + r, dc = e.dc + lane;
            if ((unsigned)dr < (unsigned)M && (unsigned)dc < (unsigned)M) {
                if (n == 255) {
                    setup[0] = 1;
                    break;
                }
                rank[(size_t)e.j * MM + rank_offset(M, R1, R2, dr, dc)] = (uint8_t)n++;
            }
        }
        cnt[ti.u0 + (ty0 + r) * ti.pitch + lane] = (uint8_t)n;
        most = max(most, n);
    }
    if (most > 0) atomicMax(setup + 1, most);
}

// out_j = conj(w) o q_j for every frame (state export of list-gather plans).
__global__ void weight_frames_kernel(int J, int MM, const float2 *q, const float2 *w, float2 *out)
{
    const size_t n = (size_t)J * MM;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        out[e] = cconjmul(__ldg(w + e % MM), q[e]);
}

// Frames of the nonblind gather slots back in frame layout (for state export).
__global__ void q_from_slots_kernel(int J, int M, int R1, int R2, const float2 *slot, const uint8_t *rank,
                                    int stride, const int32_t *frame_base, const int32_t *frame_pitch, float2 *q)
{
    const int MM = M * M;
    const size_t n = (size_t)J * MM;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / MM), k = (int)(e % MM), row = k / M, col = k % M;
        const int rk = rank[(size_t)j * MM + rank_offset(M, R1, R2, row, col)];
        q[e] = slot[(size_t)rk * stride + frame_base[j] + row * frame_pitch[j] + col];
    }
}

// u_d = R_d u0 (or 1), over the subdomain tiles
// H > 0: periodic boundaries, u0 read modulo H x W (rectangles in extended coordinates)
__device__ __forceinline__ int wrap_index(int x, int n) { const int r = x % n; return r < 0 ? r + n : r; }

__global__ void init_u_kernel(const Tile *tiles, const int32_t *rect, const int64_t *u_off, int W,
                              const float2 *u0, float2 *u, int H)
{
    const Tile tile = tiles[blockIdx.x];
    const int d = tile.reg;
    const int32_t *rc = rect + 4 * d;
    const int hd = rc[2] - rc[0], wd = rc[3] - rc[1];
    const int lane = threadIdx.x & 31, ty0 = (threadIdx.x >> 5) * TILE_ROWS;
    const int lc = tile.c0 + lane;
    if (lc >= wd) return;
    for (int r = 0; r < TILE_ROWS; ++r) {
        const int lr = tile.r0 + ty0 + r;
        if (lr >= hd) break;
        const int R = rc[0] + lr, C = rc[1] + lc;
        u[u_off[d] + (int64_t)lr * wd + lc] =
            u0 ? u0[H > 0 ? (size_t)wrap_index(R, H) * W + wrap_index(C, W) : (size_t)R * W + C]
               : make_float2(1.f, 0.f);
    }
}

__global__ void broadcast_probe_kernel(int MM, int D, const float2 *w0, float2 *w, float2 *Wd)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= MM) return;
    const float2 v = w0[k];
    w[k] = v;
    if (Wd)
        for (int d = 0; d < D; ++d) Wd[(size_t)d * MM + k] = v;
}

// The merged image at pixel (R, C): the average of the subdomain copies that
// hold it, d ascending (periodic boundaries, smax > 0: every copy (R + s_r H,
// C + s_c W), s in [-smax, smax]^2 row-major, within each d), 1 where none does.
__device__ __forceinline__ float2 merged_pixel(int R, int C, int H, int W, int D, int smax, const int32_t *rect,
                                               const int64_t *u_off, const float2 *u)
{
    float2 t = make_float2(0.f, 0.f);
    int cnt = 0;
    for (int d = 0; d < D; ++d) {
        const int32_t *rc = rect + 4 * d;
        for (int sr = -smax; sr <= smax; ++sr)
            for (int sc = -smax; sc <= smax; ++sc) {
                const int RR = R + sr * H, CC = C + sc * W;
                if (RR < rc[0] || RR >= rc[2] || CC < rc[1] || CC >= rc[3]) continue;
                t = cadd(t, u[u_off[d] + (int64_t)(RR - rc[0]) * (rc[3] - rc[1]) + (CC - rc[1])]);
                ++cnt;
            }
    }
    return cnt ? make_float2(t.x / cnt, t.y / cnt) : make_float2(1.f, 0.f);
}

// section 4: overlaps averaged, single-subdomain pixels kept
__global__ void merge_kernel(int H, int W, int D, int smax, const int32_t *rect, const int64_t *u_off,
                             const float2 *u, float2 *out)
{
    const size_t n = (size_t)H * W;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        out[e] = merged_pixel((int)(e / W), (int)(e % W), H, W, D, smax, rect, u_off, u);
}

// ---------------------------------------------------------------- peak probes
// FP32 FMA throughput: eight independent chains per thread, `iters` steps each
// (16 FLOP per thread and step); the sum goes to sink so nothing is dropped.
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, float a, float b, float *sink)
{
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (float)(threadIdx.x + i);
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
    }
    float t = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) t += x[i];
    sink[blockIdx.x * 256 + threadIdx.x] = t;
}

// Shared-memory load throughput: every step each thread reads eight 16-byte
// words, lanes on consecutive words (conflict-free), 128 bytes per thread.
__global__ void __launch_bounds__(256) smem_probe_kernel(int iters, float *sink)
{
    __shared__ float4 s[2048];
    for (int i = threadIdx.x; i < 2048; i += 256) s[i] = make_float4((float)i, 1.f, 2.f, 3.f);
    __syncthreads();
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 v = s[((warp * 8 + i + k) & 63) * 32 + lane];
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
    }
    sink[blockIdx.x * 256 + threadIdx.x] = acc.x + acc.y + acc.z + acc.w;
}

// ---------------------------------------------------------------- frame-space primal residual
// part[b] = (sum |Gamma - Gamma_snap|^2, sum sqrt(f)^2) over block b's share of
// the J m^2 frame pixels (grid-strided, fixed order); one warp finishes.
__global__ void __launch_bounds__(256) frame_residual_partial_kernel(int64_t n, const float2 *g, const float2 *g0,
                                                                     const float *sf, float *part)
{
    __shared__ float red[2 * (256 / 32)];
    float a = 0.f, b = 0.f;
    for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        a += cabs2(csub(g[i], g0[i]));
        b += sf[i] * sf[i];
    }
    block_sum2_fixed(a, b, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void frame_residual_final_kernel(int nb, const float *part, double *out)
{
    const double a = warp_sum_runs(nb, part, 2, 0);
    const double b = warp_sum_runs(nb, part, 2, 1);
    if (threadIdx.x == 0) *out = b > 0.0 ? sqrt(a / b) : 0.0;
}

// ---------------------------------------------------------------- operator norms (Lemma 2.4)
// A_d^* A_d is diagonal (eq. AtA) with entries nrm = sum_j S_j^T |w|^2, so
// ||A_d^* A_d|| = max nrm over Omega_d and ||pi_{d,e} A_d^*||^2 = max nrm over
// Omega_d n Omega_e.  Block row k < P: ordered pair k's overlap -> out[1];
// row P: every subdomain pixel -> out[0].  Maxima of non-negative floats as
// unsigned bit patterns (order-free, exact).
__global__ void __launch_bounds__(256) opnorm_kernel(int P, const int32_t *pair, const int32_t *pair_rect,
                                                     const int32_t *rect, const int64_t *u_off, int64_t u_len,
                                                     const float *nrm, uint32_t *out)
{
    const int k = blockIdx.y;
    float mx = 0.f;
    if (k < P) {
        const int d = pair[2 * k];
        const int32_t *pr = pair_rect + 4 * k, *Rd = rect + 4 * d;
        const int w = pr[3] - pr[1];
        const int64_t n = (int64_t)(pr[2] - pr[0]) * w;
        for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
            const int R = pr[0] + (int)(i / w), C = pr[1] + (int)(i % w);
            mx = fmaxf(mx, nrm[u_off[d] + (int64_t)(R - Rd[0]) * (Rd[3] - Rd[1]) + (C - Rd[1])]);
        }
    } else {
        for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < u_len; i += (int64_t)gridDim.x * 256)
            mx = fmaxf(mx, nrm[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(out + (k < P ? 1 : 0), __float_as_uint(mx));
}

// ---------------------------------------------------------------- SNR (section 4)
constexpr int SNR_BLOCKS = 152 * 4;

// Section 4's SNR of the recovery m (the merged image) against the truth t.
// pass 0: part = sum conj(m) t per block; pass 1: part = (sum |e^{i theta} m - t|^2,
// sum |m|^2) per block, e^{i theta} = ph.  Pixels where mask is 0 are left out
// (mask may be NULL).  Pixels grid-strided, fixed order.
__global__ void __launch_bounds__(256) snr_pass_kernel(int pass, int H, int W, int D, int smax, const int32_t *rect,
                                                       const int64_t *u_off, const float2 *u, const float2 *truth,
                                                       const uint8_t *mask, const double *ph, float *part)
{
    __shared__ float red[2 * (256 / 32)];
    const size_t n = (size_t)H * W;
    const float2 e = pass ? make_float2((float)ph[0], (float)ph[1]) : make_float2(1.f, 0.f);
    float a = 0.f, b = 0.f;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        if (mask && !mask[k]) continue;
        const float2 m = merged_pixel((int)(k / W), (int)(k % W), H, W, D, smax, rect, u_off, u);
        const float2 t = truth[k];
        if (pass == 0) {
            const float2 c = cconjmul(m, t);
            a += c.x;
            b += c.y;
        } else {
            const float2 em = make_float2(e.x * m.x - e.y * m.y, e.x * m.y + e.y * m.x);
            a += cabs2(csub(em, t));
            b += cabs2(m);
        }
    }
    block_sum2_fixed(a, b, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

// pass 0: out[0..1] = e^{i theta}, theta = arg sum conj(m) t; pass 1: out[2] = SNR (dB).
// One warp, fixed order.
__global__ void snr_final_kernel(int pass, const float *part, double *out)
{
    const double a = warp_sum_runs(SNR_BLOCKS, part, 2, 0);
    const double b = warp_sum_runs(SNR_BLOCKS, part, 2, 1);
    if (threadIdx.x != 0) return;
    if (pass == 0) {
        const double r = sqrt(a * a + b * b);
        out[0] = r > 0.0 ? a / r : 1.0;
        out[1] = r > 0.0 ? b / r : 0.0;
    } else {
        out[2] = -10.0 * log10(a / b);
    }
}

__global__ void prox_kernel(const float2 *y, const float *f, float2 *z, int64_t n, float lam,
                            float inv1plam, float c_thr, float c_k1)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 yv = y[i];
        const float sf = sqrtf(fmaxf(f[i], 0.f));
        const float ay = sqrtf(yv.x * yv.x + yv.y * yv.y);
        float rho;
        if (ay < c_thr * sf)
            rho = fmaxf(0.f, c_k1 * ay);
        else
            rho = (sf + lam * ay) * inv1plam;
        float2 out;
        if (ay > 0.f) {
            const float s = rho / ay;
            out = make_float2(yv.x * s, yv.y * s);
        } else {
            out = make_float2(rho, 0.f);
        }
        z[i] = out;
    }
}

// ---- data-driven initial probe (section 4.2): w0 = (1/J) sum_j F^* sqrt(f_j),
// formed as F^* of the mean amplitude (the inverse DFT is linear).

// Mean measured amplitude per frequency, natural order.  One thread per stored
// element (coalesced over frames); the J frames are added in ascending j with
// compensated (Kahan) FP32 addition.  Storage index s holds position (pr, pc)
// at s = pc m + pr (transposed) or pr m + pc (row_major); position p holds
// frequency p / R2 + R1 (p % R2).
__global__ void amp_mean_kernel(int J, int M, int R1, int R2, int row_major, const float *__restrict__ sqrtf_,
                                float *__restrict__ amp)
{
    const int MM = M * M;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < MM; s += gridDim.x * blockDim.x) {
        float sum = 0.f, c = 0.f;
        for (int j = 0; j < J; ++j) {
            const float y = sqrtf_[(size_t)j * MM + s] - c;
            const float t = sum + y;
            c = (t - sum) - y;
            sum = t;
        }
        const int a = s / M, b = s % M;
        const int pr = row_major ? a : b, pc = row_major ? b : a;
        const int kr = pr / R2 + R1 * (pr % R2), kc = pc / R2 + R1 * (pc % R2);
        amp[kr * M + kc] = sum / (float)J;
    }
}

// T[kr][c] = sum_kc amp[kr][kc] exp(+2 pi i kc c / M) (direct sum, kc ascending)
__global__ void idft_rows_kernel(int M, const float *__restrict__ amp, const float2 *__restrict__ tw,
                                 float2 *__restrict__ T)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * M) return;
    const int kr = e / M, c = e % M;
    float2 acc = make_float2(0.f, 0.f);
    for (int kc = 0; kc < M; ++kc) {
        const float2 t = tw[(kc * c) % M];  // exp(-2 pi i kc c / M); conjugated below
        const float v = amp[kr * M + kc];
        acc.x += v * t.x;
        acc.y -= v * t.y;
    }
    T[e] = acc;
}

// w0[r][c] = (1/M) sum_kr T[kr][c] exp(+2 pi i kr r / M) (kr ascending)
__global__ void idft_cols_kernel(int M, const float2 *__restrict__ T, const float2 *__restrict__ tw,
                                 float2 *__restrict__ w0)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * M) return;
    const int r = e / M, c = e % M;
    float2 acc = make_float2(0.f, 0.f);
    for (int kr = 0; kr < M; ++kr) {
        const float2 t = tw[(kr * r) % M];
        const float2 v = T[kr * M + c];
        acc.x += v.x * t.x + v.y * t.y;  // v * conj(t)
        acc.y += v.y * t.x - v.x * t.y;
    }
    w0[e] = make_float2(acc.x / (float)M, acc.y / (float)M);
}

}  // namespace

void fill_sub_args(const ptycho_plan_s *p, SubArgs out[2])
{
    for (int par = 0; par < 2; ++par) {
        SubArgs &a = out[par];
        a = SubArgs{};
        a.M = p->M;
        a.rect = p->d_rect;
        a.u_off = p->d_u_off;
        a.tinfo = p->sub_tiles.info;
        a.tlist = p->sub_tiles.list;
        a.tnbr = p->sub_tiles.nbr;
        a.u_cur = p->d_u[par];
        a.lam_cur = p->d_lam[par];
        a.u_next = p->d_u[1 - par];
        a.lam_next = p->d_lam[1 - par];
        a.q = p->d_q;
        a.w = p->d_w;
        // list gather (blind, or nonblind without slots): weight with W_d, or
        // with the known probe for every subdomain
        a.Wd = p->blind ? p->d_Wd : p->d_w;
        a.wd_stride = p->blind ? p->MM : 0;
        a.nrm = p->d_nrm;
        a.slot = p->d_slot;
        a.cnt = p->d_cnt;
        a.slot_stride = (int32_t)p->u_len;
        a.eta = p->eta;
        a.r = p->r;
        a.gamma = p->blind ? p->gamma : 0.f;
        a.blind = p->blind;
        a.re_part = p->d_re_part;
    }
}

int launch_subdomain_update_table(bool blind, const SubArgs *tab, const int2 *items, int n_items, int parity,
                                  cudaStream_t s)
{
    if (n_items <= 0) return PTYCHO_OK;
    if (blind)
        subdomain_update_kernel<true, true><<<n_items, GATHER_THREADS, 0, s>>>(SubArgs{}, tab, items, parity);
    else
        subdomain_update_kernel<false, true><<<n_items, GATHER_THREADS, 0, s>>>(SubArgs{}, tab, items, parity);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_subdomain_update(ptycho_plan_s *p, cudaStream_t s)
{
    const int n = p->sub_tiles.n_tiles;
    if (n <= 0) return PTYCHO_OK;
    if (p->blind || !p->slots)
        subdomain_update_kernel<true, false><<<n, GATHER_THREADS, 0, s>>>(p->h_sargs[p->cur], nullptr, nullptr, p->cur);
    else
        subdomain_update_kernel<false, false><<<n, GATHER_THREADS, 0, s>>>(p->h_sargs[p->cur], nullptr, nullptr, p->cur);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_image_gather(const ptycho_plan_s *p, const float2 *q, const float2 *w, float2 *out,
                        cudaStream_t s)
{
    image_gather_kernel<<<p->img_tiles.n_tiles, GATHER_THREADS, 0, s>>>(
        p->M, p->img_rows, p->img_cols, p->img_tiles.tiles, p->img_tiles.ptr, p->img_tiles.list, q, w, out);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

__global__ void wrap_pad_kernel(int H, int W, int Hp, int Wp, const float2 *__restrict__ u, float2 *__restrict__ up)
{
    const size_t n = (size_t)Hp * Wp;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int R = (int)(e / Wp), C = (int)(e % Wp);
        up[e] = u[(size_t)(R < H ? R : R - H) * W + (C < W ? C : C - W)];
    }
}

// each image pixel: its copies in the padded grid added in a fixed order
__global__ void fold_kernel(int H, int W, int Hp, int Wp, const float2 *__restrict__ gp, float2 *__restrict__ out)
{
    const size_t n = (size_t)H * W;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int R = (int)(e / W), C = (int)(e % W);
        float2 t = gp[(size_t)R * Wp + C];
        if (C + W < Wp) t = cadd(t, gp[(size_t)R * Wp + C + W]);
        if (R + H < Hp) {
            t = cadd(t, gp[(size_t)(R + H) * Wp + C]);
            if (C + W < Wp) t = cadd(t, gp[(size_t)(R + H) * Wp + C + W]);
        }
        out[e] = t;
    }
}

int launch_wrap_pad(const ptycho_plan_s *p, const float2 *u, cudaStream_t s)
{
    wrap_pad_kernel<<<152 * 8, 256, 0, s>>>(p->H, p->W, p->img_rows, p->img_cols, u, p->d_upad);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_fold(const ptycho_plan_s *p, float2 *out, cudaStream_t s)
{
    fold_kernel<<<152 * 8, 256, 0, s>>>(p->H, p->W, p->img_rows, p->img_cols, p->d_gpad, out);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

// grad_w == nullptr: blind W-update over the subdomain groups (u = current
// subdomain buffer, h = d_q).  Otherwise: grad_w = sum over all frames of
// conj(S_j u_img) h_j (one group).
int launch_probe_reduce(ptycho_plan_s *p, const float2 *u_img, float2 *grad_w, cudaStream_t s, const float2 *h)
{
    const od2p::ProbeGroups &G = grad_w ? p->img_groups : p->sub_groups;
    ProbeArgs a;
    a.M = p->M;
    a.chunks = G.chunks;
    a.group_frames = G.frames;
    a.frame_base = grad_w ? p->d_img_base : p->d_frame_base;
    a.frame_pitch = grad_w ? nullptr : p->d_frame_pitch;
    a.pitch = p->img_cols;
    a.u = grad_w ? u_img : p->d_u[p->cur];
    a.h = h ? h : p->d_q;
    a.part = p->d_probe_part;
    a.part_n = p->d_probe_part_n;
    const int MM = p->MM;
    if (G.n_chunks > 0) {
        dim3 grid((MM + 255) / 256, G.n_chunks);
        probe_partial_kernel<<<grid, 256, 0, s>>>(a);
        OD2P_CUDA(cudaGetLastError());
    }
    if (grad_w) {
        probe_finalize_sum_kernel<<<(MM + 255) / 256, 256, 0, s>>>(p->M, G.n_chunks, p->d_probe_part, grad_w);
    } else {
        dim3 grid((MM + 255) / 256, p->D);
        probe_finalize_blind_kernel<<<grid, 256, 0, s>>>(p->M, p->D, G.chunk_ptr, p->d_probe_part,
                                                         p->d_probe_part_n, p->d_wnew, p->d_Wd,
                                                         p->d_Delta, p->eta, p->mu);
    }
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

// Halo rows of a shard: one warp per row, lanes along the row (coalesced).
__global__ void halo_copy_kernel(const HaloRow *rows, int n_rows, float2 *u, float2 *lam, float2 *Wd,
                                 float2 *Delta, float2 *msg, int pack)
{
    const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (row >= n_rows) return;
    const HaloRow r = rows[row];
    float2 *a = r.arr == 0 ? u : r.arr == 1 ? lam : r.arr == 2 ? Wd : Delta;
    if (pack)
        for (int i = lane; i < r.len; i += 32) msg[r.msg + i] = a[r.off + i];
    else
        for (int i = lane; i < r.len; i += 32) a[r.off + i] = msg[r.msg + i];
}

int launch_halo_copy(const ptycho_plan_s *p, const HaloRow *rows, int n_rows, float2 *msg, bool pack,
                     cudaStream_t s)
{
    if (n_rows <= 0) return PTYCHO_OK;
    const int blocks = (n_rows + 7) / 8;  // eight warps per block
    halo_copy_kernel<<<blocks, 256, 0, s>>>(rows, n_rows, p->d_u[p->cur], p->d_lam[p->cur], p->d_Wd, p->d_Delta, msg,
                                            pack ? 1 : 0);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_loss_reduce(ptycho_plan_s *p, float *loss, cudaStream_t s)
{
    loss_sum_kernel<<<1, 256, 0, s>>>(p->n_loss_blocks, p->d_loss_part, loss);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_probe_init(ptycho_plan_s *p, float2 *w0, cudaStream_t s)
{
    int R1 = 1, R2 = 256, row_major = 1;  // m = 256: natural order (k = p)
    if (p->M != 256) {
        rank_radix(p->M, &R1, &R2);  // m <= 128: transposed position layout
        row_major = 0;
    }
    float *amp = reinterpret_cast<float *>(p->d_q);  // plan scratch: MM floats
    float2 *T = p->d_wnew;                           // plan scratch: MM complex
    const int blocks = (p->MM + 255) / 256;
    amp_mean_kernel<<<blocks, 256, 0, s>>>(p->J, p->M, R1, R2, row_major, p->d_sqrtf, amp);
    OD2P_CUDA(cudaGetLastError());
    idft_rows_kernel<<<blocks, 256, 0, s>>>(p->M, amp, p->d_tw, T);
    OD2P_CUDA(cudaGetLastError());
    idft_cols_kernel<<<blocks, 256, 0, s>>>(p->M, T, p->d_tw, w0);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_scale(float2 *x, int64_t n, float sc, cudaStream_t s)
{
    if (n <= 0) return PTYCHO_OK;
    scale_kernel<<<152 * 8, 256, 0, s>>>(n, x, sc);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_consensus(ptycho_plan_s *p, float *part, double *out, cudaStream_t s)
{
    consensus_partial_kernel<<<dim3(RC_BLOCKS, p->P + 1), 256, 0, s>>>(p->P, p->d_pair, p->d_pair_rect,
                                                                        p->periodic ? p->d_pair_shift : nullptr,
                                                                        p->H, p->W, p->d_rect,
                                                                        p->d_u_off, p->u_len, p->d_u[p->cur], part);
    OD2P_CUDA(cudaGetLastError());
    consensus_final_kernel<<<1, 32, 0, s>>>(p->P, part, out);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_metrics(ptycho_plan_s *p, cudaStream_t s)
{
    metrics_kernel<<<1, 1024, 0, s>>>(p->n_rf_parts, p->d_rf_part, p->D, p->sub_tiles.reg_ptr,
                                    p->d_re_part, p->d_metrics);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_sum_sqrtf(ptycho_plan_s *p, cudaStream_t s)
{
    sum_kernel<<<1, 256, 0, s>>>(p->J, p->d_loss_part, p->d_metrics + 2);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_init_state(ptycho_plan_s *p, const float2 *u0, const float2 *w0, cudaStream_t s)
{
    init_u_kernel<<<p->sub_tiles.n_tiles, GATHER_THREADS, 0, s>>>(p->sub_tiles.tiles, p->d_rect,
                                                                  p->d_u_off, p->W, u0, p->d_u[p->cur],
                                                                  p->periodic ? p->H : 0);
    OD2P_CUDA(cudaGetLastError());
    broadcast_probe_kernel<<<(p->MM + 255) / 256, 256, 0, s>>>(p->MM, p->D, w0, p->d_w,
                                                                p->blind ? p->d_Wd : nullptr);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_illumination(ptycho_plan_s *p, cudaStream_t s)
{
    illumination_kernel<<<p->sub_tiles.n_tiles, GATHER_THREADS, 0, s>>>(
        p->M, p->d_rect, p->d_u_off, p->sub_tiles.tiles, p->sub_tiles.ptr, p->sub_tiles.list, p->d_w, p->d_nrm);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_slot_rank(ptycho_plan_s *p, int32_t *setup, cudaStream_t s)
{
    int R1 = 0, R2 = 0;
    rank_radix(p->M, &R1, &R2);
    slot_rank_kernel<<<p->sub_tiles.n_tiles, GATHER_THREADS, 0, s>>>(p->M, R1, R2, p->sub_tiles.info,
                                                                      p->sub_tiles.list, p->d_rank, p->d_cnt, setup);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_q_from_slots(const ptycho_plan_s *p, float2 *dst, cudaStream_t s)
{
    if (!p->slots) {  // list-gather plans keep q unweighted: apply conj(w) here
        weight_frames_kernel<<<152 * 8, 256, 0, s>>>(p->J, p->MM, p->d_q, p->d_w, dst);
        OD2P_CUDA(cudaGetLastError());
        return PTYCHO_OK;
    }
    int R1 = 0, R2 = 0;
    rank_radix(p->M, &R1, &R2);
    q_from_slots_kernel<<<152 * 8, 256, 0, s>>>(p->J, p->M, R1, R2, p->d_slot, p->d_rank, (int)p->u_len, p->d_frame_base,
                                               p->d_frame_pitch, dst);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_merge(const ptycho_plan_s *p, float2 *out, cudaStream_t s)
{
    merge_kernel<<<152 * 8, 256, 0, s>>>(p->H, p->W, p->D, p->periodic ? PERIOD_SHIFTS : 0, p->d_rect, p->d_u_off,
                                         p->d_u[p->cur], out);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_peak_probe(int kind, int n_blocks, int iters, float *sink, cudaStream_t s)
{
    if (kind == 0)
        fma_probe_kernel<<<n_blocks, 256, 0, s>>>(iters, 0.999999f, 1e-7f, sink);
    else
        smem_probe_kernel<<<n_blocks, 256, 0, s>>>(iters, sink);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_until_init(int32_t *st, int32_t max_iter, float tol, cudaStream_t s)
{
    until_init_kernel<<<1, 1, 0, s>>>(st, max_iter, tol);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

// Does a device-set condition take effect?  A graph whose if-node (default 0)
// guards a marking kernel, the condition set to 1 by a kernel before it; no
// loop, so nothing can spin.  *ok = 1 when the body ran.
int conditional_selftest(int32_t *scratch, int *ok, cudaStream_t s)
{
    *ok = 0;
    cudaGraph_t G = nullptr;
    cudaGraphExec_t X = nullptr;
    cudaError_t e = cudaSuccess;
    auto done = [&](int code) {
        if (X) cudaGraphExecDestroy(X);
        if (G) cudaGraphDestroy(G);
        return code;
    };
    if ((e = cudaGraphCreate(&G, 0)) != cudaSuccess) return done(cuda_fail(e, "cudaGraphCreate"));
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, G, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
        return done(cuda_fail(e, "cudaGraphConditionalHandleCreate"));
    unsigned one = 1u;
    void *set_args[] = {&h, &one};
    cudaKernelNodeParams kp = {};
    kp.func = reinterpret_cast<void *>(cond_set_kernel);
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = set_args;
    cudaGraphNode_t set_node, if_node, mark_node;
    if ((e = cudaGraphAddKernelNode(&set_node, G, nullptr, 0, &kp)) != cudaSuccess)
        return done(cuda_fail(e, "cudaGraphAddKernelNode"));
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = h;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    if ((e = cudaGraphAddNode(&if_node, G, &set_node, nullptr, 1, &ip)) != cudaSuccess)
        return done(cuda_fail(e, "cudaGraphAddNode (if)"));
    void *mark_args[] = {&scratch};
    kp.func = reinterpret_cast<void *>(cond_mark_kernel);
    kp.kernelParams = mark_args;
    if ((e = cudaGraphAddKernelNode(&mark_node, ip.conditional.phGraph_out[0], nullptr, 0, &kp)) != cudaSuccess)
        return done(cuda_fail(e, "cudaGraphAddKernelNode"));
    if ((e = cudaGraphInstantiate(&X, G, 0)) != cudaSuccess) return done(cuda_fail(e, "cudaGraphInstantiate"));
    int32_t h_flag = 0;
    if ((e = cudaMemsetAsync(scratch, 0, sizeof(int32_t), s)) != cudaSuccess ||
        (e = cudaGraphLaunch(X, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&h_flag, scratch, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return done(cuda_fail(e, "conditional self check"));
    *ok = h_flag == 1;
    return done(PTYCHO_OK);
}

// Kernel node of the stopping test (arguments copied by the graph at creation).
int add_until_check_node(cudaGraphNode_t *node, cudaGraph_t graph, const cudaGraphNode_t *dep, ptycho_plan_s *p,
                         cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_second, int set_second)
{
    int n_rf = p->n_rf_parts;
    const float *rf_part = p->d_rf_part;
    const double *metrics = p->d_metrics;
    int32_t *st = p->d_until;
    void *args[] = {&n_rf, &rf_part, &metrics, &st, &h_loop, &h_second, &set_second};
    cudaKernelNodeParams kp = {};
    kp.func = reinterpret_cast<void *>(until_check_kernel);
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1024);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    OD2P_CUDA(cudaGraphAddKernelNode(node, graph, dep, dep ? 1 : 0, &kp));
    return PTYCHO_OK;
}

int launch_frame_residual(ptycho_plan_s *p, const float2 *snap, float *part, double *out, cudaStream_t s)
{
    constexpr int NB = SNR_BLOCKS;  // the SNR partial buffer holds 2 x SNR_BLOCKS floats
    frame_residual_partial_kernel<<<NB, 256, 0, s>>>((int64_t)p->J * p->MM, p->d_gamma, snap, p->d_sqrtf, part);
    OD2P_CUDA(cudaGetLastError());
    frame_residual_final_kernel<<<1, 32, 0, s>>>(NB, part, out);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_operator_norms(ptycho_plan_s *p, uint32_t *out, cudaStream_t s)
{
    OD2P_CUDA(cudaMemsetAsync(out, 0, 2 * sizeof(uint32_t), s));
    opnorm_kernel<<<dim3(RC_BLOCKS, p->P + 1), 256, 0, s>>>(p->P, p->d_pair, p->d_pair_rect, p->d_rect, p->d_u_off,
                                                            p->u_len, p->d_nrm, out);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

int launch_snr(ptycho_plan_s *p, const float2 *truth, const uint8_t *mask, float *part, double *out,
               cudaStream_t s)
{
    for (int pass = 0; pass < 2; ++pass) {
        snr_pass_kernel<<<SNR_BLOCKS, 256, 0, s>>>(pass, p->H, p->W, p->D, p->periodic ? PERIOD_SHIFTS : 0,
                                                   p->d_rect, p->d_u_off, p->d_u[p->cur],
                                                   truth, mask, out, part);
        OD2P_CUDA(cudaGetLastError());
        snr_final_kernel<<<1, 32, 0, s>>>(pass, part, out);
        OD2P_CUDA(cudaGetLastError());
    }
    return PTYCHO_OK;
}

int launch_prox(const float2 *y, const float *f, float2 *z, int64_t n, float eps, float lam,
                cudaStream_t s)
{
    const float c_thr = eps - (1.f - eps) / lam;
    const float c_k1 = c_thr > 0.f ? lam / (lam - (1.f - eps) / eps) : 0.f;
    const int64_t blocks = (n + 255) / 256;
    prox_kernel<<<(int)(blocks < 152 * 32 ? blocks : 152 * 32), 256, 0, s>>>(
        y, f, z, n, lam, 1.f / (1.f + lam), c_thr, c_k1);
    OD2P_CUDA(cudaGetLastError());
    return PTYCHO_OK;
}

}  // namespace od2p
