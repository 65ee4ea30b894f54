// Internal declarations of the sm_103a OD2P library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/od2p.h"

namespace od2p {

// Thread block tile of the gather kernels: TILE_H rows x TILE_W columns.
// Lanes run along a row (coalesced frame rows); each thread owns TILE_ROWS
// consecutive rows of its column, so one frame-list entry drives TILE_ROWS
// independent loads.
#ifndef OD2P_TILE_H
#define OD2P_TILE_H 32
#endif
constexpr int TILE_H = OD2P_TILE_H;
constexpr int TILE_W = 32;
constexpr int GATHER_THREADS = 256;
constexpr int TILE_ROWS = TILE_H * TILE_W / GATHER_THREADS;
// Frames per chunk of the fixed-order probe reductions (blind W, grad w).
#ifndef OD2P_PROBE_CHUNK
#define OD2P_PROBE_CHUNK 32
#endif
constexpr int PROBE_CHUNK = OD2P_PROBE_CHUNK;
// m = 256 frames go through their three FFT passes in waves of this many
// frames (a 10 MB intermediate per wave that stays in L2), with up to
// WAVE_CHAINS_256 waves in flight side by side: the default shape of a plan,
// which ptycho_plan_set_waves changes (up to MAX_WAVE_CHAINS chains of at most
// MAX_WAVE_FRAMES frames).
#ifndef OD2P_WAVE_256
#define OD2P_WAVE_256 19
#endif
constexpr int WAVE_256 = OD2P_WAVE_256;
#ifndef OD2P_WAVE_CHAINS_256
#define OD2P_WAVE_CHAINS_256 4
#endif
constexpr int WAVE_CHAINS_256 = OD2P_WAVE_CHAINS_256;
constexpr int MAX_WAVE_CHAINS = 8, MAX_WAVE_FRAMES = 152;
static_assert(WAVE_CHAINS_256 >= 1 && WAVE_CHAINS_256 <= MAX_WAVE_CHAINS && WAVE_256 >= 1 &&
                  WAVE_256 <= MAX_WAVE_FRAMES, "default wave shape");
// Periodic boundaries: rectangles inside (-H, 2H) x (-W, 2W) meet copies of each
// other shifted by at most this many periods per axis.
constexpr int PERIOD_SHIFTS = 2;

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define OD2P_CUDA(call)                                                     \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return ::od2p::cuda_fail(e_, #call);         \
    } while (0)

// Tile of a gather: pixel block [r0, r0+TILE_H) x [c0, c0+TILE_W) of region
// `reg` (a subdomain, or the whole image), and the frames that intersect it
// in ascending j: list[ptr_begin, ptr_end).
struct Tile {
    int32_t reg, r0, c0, pad;
};

// Entry of a tile's frame list: frame j and the tile origin relative to the
// window origin (tile_row0 - o_r, tile_col0 - o_c), so that a pixel at
// (ty, tx) of the tile reads frame pixel (dr + ty, dc + tx).
struct ListEntry {
    int32_t j, dr, dc, pad;
};

struct NbrInfo;

// Everything the subdomain update needs about one tile of a subdomain, read
// with one 48-byte load: u index of the tile's first pixel and the row pitch
// of u_d, the tile's extent inside Omega_d, its image coordinates, its
// neighbour and frame-list ranges, its subdomain and the last row of Omega_d.
struct TileInfo {
    int32_t u0, pitch, nrows, ncols;
    int32_t R0, C0, n0, nnb;
    int32_t k0, nk, reg, rend;
};

struct GatherTiles {
    int32_t n_tiles = 0;
    Tile *tiles = nullptr;        // device
    int32_t *ptr = nullptr;       // device, n_tiles + 1
    ListEntry *list = nullptr;    // device
    int32_t *reg_ptr = nullptr;   // device, first tile of each region (+ end)
    int32_t *nbr_ptr = nullptr;   // device, n_tiles + 1: neighbours meeting the tile
    NbrInfo *nbr = nullptr;       // device
    TileInfo *info = nullptr;     // device, n_tiles (subdomain tiles only)
};

// A neighbour e of subdomain d, precomputed for the subdomain update.
struct NbrInfo {
    int32_t r0, c0, r1, c1;       // Omega_e
    int32_t u_base, u_pitch;      // u_e storage: index of (r0, c0), row pitch
    int32_t p_r0, p_c0, p_pitch;  // Omega_d n Omega_e: origin and row pitch of Lambda storage
    int32_t lam_de, lam_ed;       // offsets of Lambda_{d,e} and Lambda_{e,d}
    int32_t d_first;              // 1 if d < e (fixes the operand order of v)
};

// Frame groups of the fixed-order probe reductions, cut into chunks of
// PROBE_CHUNK frames: chunk c covers frames[begin, end) of group `group`.
struct ProbeGroups {
    int32_t n_groups = 0, n_chunks = 0;
    int32_t *frames = nullptr;    // device, frame ids ascending within a group
    int4 *chunks = nullptr;       // device, (group, begin, end, 0)
    int32_t *chunk_ptr = nullptr; // device, first chunk of each group (+ end)
};

// ST-AGM prox constants for lambda (eq. Prox_sol with the threshold read as
// |y| < (eps - (1-eps)/lambda) sqrt f).
struct ProxConst {
    float lam, inv1plam, c_thr, c_k1;
};

inline ProxConst make_prox_const(float eps, float lam)
{
    ProxConst k;
    k.lam = lam;
    k.inv1plam = 1.f / (1.f + lam);
    k.c_thr = eps - (1.f - eps) / lam;
    k.c_k1 = k.c_thr > 0.f ? lam / (lam - (1.f - eps) / eps) : 0.f;
    return k;
}

// Arguments of one plan's frame update (one copy per buffer parity), read by
// the persistent frame-update kernel from a device table so that one launch
// can serve several plans.
struct FrameArgs {
    int32_t J;
    const int32_t *frame_sub, *frame_base, *frame_pitch;
    const float2 *u, *w, *Wd; // Wd non-null for blind plans (per-subdomain probe)
    float2 *gamma;            // transposed position layout
    const float *sqrtf_;      // transposed position layout
    float2 *q;                // out (blind): F^*(z - Gamma^{n+1}), natural spatial order
    float2 *slot;             // out (nonblind): conj(w) o F^*(z - Gamma^{n+1}) in gather slots
    const uint8_t *rank;      // nonblind: slot rank of each frame pixel
    int32_t slot_stride;      // u_len
    float *rf_part;           // out: one partial per frame group
    int32_t *err;             // set to 1 if a pipeline wait gives up
    const float2 *tw;
    ProxConst pc;
};

// One row of a halo message: `len` elements of array `arr` (0: u, 1: Lambda,
// 2: W_d, 3: Delta_d) from offset `off`, at offset `msg` of the message.
struct HaloRow {
    int32_t arr, len;
    int64_t off, msg;
};

// Arguments of one plan's subdomain update (one copy per buffer parity).
struct SubArgs {
    int32_t M;
    const int32_t *rect;
    const int64_t *u_off;
    const TileInfo *tinfo;
    const ListEntry *tlist;
    const NbrInfo *tnbr;
    const float2 *u_cur, *lam_cur, *q, *w, *Wd;
    const float *nrm;
    const float2 *slot;        // nonblind gather slots
    const uint8_t *cnt;
    int32_t slot_stride;
    float2 *u_next, *lam_next;
    float eta, r, gamma;
    int32_t blind;
    int32_t wd_stride;         // list gather: probe of tile subdomain d at Wd + d * wd_stride
    float *re_part;
};

}  // namespace od2p

struct ptycho_plan_s {
    // ---- problem
    int32_t H = 0, W = 0, M = 0, MM = 0, J = 0, D = 0, P = 0;
    int32_t sub_rows = 0, sub_cols = 0, overlap_px = 0;
    float eps = 0, eta = 0, r = 0, mu = 0, gamma = 0;
    int32_t blind = 0;
    bool has_mask = false;
    bool periodic = false;         // periodic boundaries: rectangles in extended coordinates
    // whole-image windows (forward operator, loss, adjoint): the image itself
    // (img_rows x img_cols = H x W), or for periodic plans a wrapped copy of
    // (H + m - 1) x (W + m - 1) pixels in which no window wraps
    int32_t img_rows = 0, img_cols = 0;
    float2 *d_upad = nullptr, *d_gpad = nullptr;  // periodic: the wrapped image, the adjoint before folding
    // ---- host copies of the decomposition (offs: each frame's placed offset)
    std::vector<int32_t> offs, frame_sub, rect, pair, pair_rect, pair_shift;
    std::vector<int64_t> u_off, lam_off;
    int64_t u_len = 0, lam_len = 0;
    // ---- device geometry
    int32_t *d_offs = nullptr, *d_frame_sub = nullptr, *d_frame_base = nullptr,
            *d_frame_pitch = nullptr, *d_rect = nullptr, *d_nbr_ptr = nullptr, *d_nbr = nullptr,
            *d_pair_rect = nullptr, *d_pair = nullptr, *d_img_base = nullptr,  // nbr: (e, pair d-e, pair e-d) per neighbour
            *d_pair_shift = nullptr,                     // (s_r, s_c) per pair, in periods
            *d_img_pitch = nullptr;                      // img_w for every frame
    od2p::NbrInfo *d_nbr_info = nullptr;  // per neighbour entry, same order as d_nbr
    int64_t *d_u_off = nullptr, *d_lam_off = nullptr;
    od2p::GatherTiles sub_tiles, img_tiles;
    od2p::ProbeGroups sub_groups, img_groups;
    float2 *d_tw = nullptr;        // M twiddles exp(-2 pi i k / M)
    float *d_mask = nullptr;       // M*M Fourier support (blind), or null
    // ---- device state (Gamma and sqrt f in the frame kernel's transposed layout)
    float *d_sqrtf = nullptr;      // J*MM
    float2 *d_gamma = nullptr;     // J*MM
    float2 *d_q = nullptr;         // J*MM frame residuals / scratch
    float2 *d_T = nullptr;         // m = 256: t_waves x wave_frames frames of FFT intermediate
    int64_t t_cap_frames = 0;      // m = 256: frames d_T holds
    int32_t wave_frames = 0;       // m = 256: frames per wave
    int32_t t_waves = 1;           // m = 256: chains of waves in flight
    cudaStream_t wave_stream[od2p::MAX_WAVE_CHAINS] = {};  // m = 256: streams of chains 1 .. (made on demand)
    cudaEvent_t wave_ev[od2p::MAX_WAVE_CHAINS] = {};       // [0] fork, [c] join of chain c
    // Nonblind gather slots: frame j's weighted residual at window pixel k goes to
    // d_slot[rank_j(k) * u_len + (index of that pixel in the u buffer)], where
    // rank_j(k) counts the frames of the subdomain with smaller index that cover
    // the same pixel; d_cnt holds each subdomain pixel's number of frames.
    uint8_t *d_rank = nullptr;     // J*MM
    uint8_t *d_cnt = nullptr;      // u_len
    float2 *d_slot = nullptr;      // slot_k * u_len
    int32_t slot_k = 0;
    // nonblind plans gather through slots unless more than 255 frames cover a
    // pixel or the slots would exceed 2^32 elements; then they take the
    // frame-list gather of blind plans, weighting with the known probe
    bool slots = false;
    float2 *d_u[2] = {nullptr, nullptr};
    float *d_nrm = nullptr;        // nonblind: sum_j S_j^T |w|^2 per subdomain pixel (eq. AtA)
    float2 *d_lam[2] = {nullptr, nullptr};
    float2 *d_w = nullptr, *d_wnew = nullptr, *d_Wd = nullptr, *d_Delta = nullptr;
    float2 *d_probe_part = nullptr;    // blind / grad-w partial sums
    float *d_probe_part_n = nullptr;
    float *d_rf_part = nullptr;        // one per frame-kernel block
    float *d_re_part = nullptr;        // 2 per subdomain tile
    float *d_loss_part = nullptr;
    double *d_metrics = nullptr;       // [rf, re, sum sqrt f, consensus residual, loss (float)]
    float *d_rc_part = nullptr;        // (P + 1) x 64 partial sums of the consensus residual
    float *d_snr_part = nullptr;       // 2 x 608 partial sums of the SNR passes
    double *d_snr = nullptr;           // [cos theta, sin theta, SNR dB]
    uint32_t *d_opn = nullptr;         // operator norms as float bits: [max A^*A, max over overlaps]
    int32_t *d_err = nullptr;          // set by a kernel whose bounded wait gave up
    int32_t n_k1_blocks = 0;           // blocks of the persistent frame update
    int32_t k1_variant = 0;            // launch shape of the frame update (0 or 1)
    int32_t k1_blocks_per_sm = 0;      // resident-block cap of the frame update (0: as many as fit)
    bool batch_member = false;         // owned by a batch, which sets its launch shape
    int32_t n_rf_parts = 0;            // RF partial sums (one per warp of each frame group / m = 256 slab)
    od2p::FrameArgs h_fargs[2];        // frame-update arguments by buffer parity
    od2p::SubArgs h_sargs[2];          // subdomain-update arguments by buffer parity
    od2p::FrameArgs *d_fargs = nullptr;
    od2p::SubArgs *d_sargs = nullptr;
    int32_t n_loss_blocks = 0;         // blocks of the loss kernel
    int32_t cur = 0;                   // which u / Lambda buffer holds the current iterate
    bool initialised = false;
    // ---- graphs
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t until[2] = {nullptr, nullptr};  // iterate-until loops, by starting parity
    int32_t *d_until = nullptr;                      // [done, cap, tol bits, last RF bits]
    bool cond_checked = false;                       // conditional-node self check passed
    int32_t fft_kind = 0;                            // m = 64: 0 the 8 x 8 split, 1 / 2 the 16 x 4 split
    float2 *d_gamma_snap = nullptr;                  // Gamma snapshot (allocated on first use)
    // stagm_loss_grad's stored gradient frames (recompute = 0 stores, 2 reuses)
    float2 *d_hstore = nullptr;                      // J*MM, allocated on first store
    float *d_hloss = nullptr;                        // the loss of the stored pass
    const void *h_u = nullptr, *h_w = nullptr;       // the u and w it was computed from
    bool h_stored = false;
    // ---- shards (ptycho_plan_shard): the subdomains of rank `rank` of `world`
    std::vector<int32_t> global_j;   // global index of each of the plan's frames
    std::vector<int32_t> owner;      // D: owning rank of each subdomain (empty: not a shard)
    int32_t rank = 0, world = 1;
    struct Halo {                    // messages to / from one peer
        int64_t send_n = 0, recv_n = 0;
        int32_t send_rows = 0, recv_rows = 0;
        od2p::HaloRow *d_send = nullptr, *d_recv = nullptr;
    };
    std::vector<Halo> halo;          // by peer rank
    // ---- every device allocation, freed by ptycho_plan_destroy
    std::vector<void *> owned;
};

namespace od2p {

// fft_kernels.cu
int launch_frame_update(ptycho_plan_s *p, cudaStream_t s);
int f4_grid(int kind, int J, int *grid, int blocks_per_sm = 0);
int launch_frame_update_f4_table(const FrameArgs *tab, const int2 *items, int n_items, int grid, int parity,
                                 cudaStream_t s);
int launch_forward(const ptycho_plan_s *p, const float2 *u, const float2 *w, float2 *out,
                   cudaStream_t s);
int launch_frames_ifft_weight(const ptycho_plan_s *p, const float2 *frames, const float2 *w,
                              bool ifft, float2 *out, cudaStream_t s);
// h_j = F^* grad g of every frame into h_out (null: the plan's frame scratch) and loss partials
int launch_loss_frames(ptycho_plan_s *p, const float2 *u, const float2 *w, cudaStream_t s, float2 *h_out = nullptr);
// ST-AGM loss partials of the current subdomain iterate (u_d, and W_d when blind)
int launch_metrics_loss(ptycho_plan_s *p, cudaStream_t s);
int launch_probe_avg(ptycho_plan_s *p, cudaStream_t s);
int launch_ingest_f(ptycho_plan_s *p, const float *f, cudaStream_t s);
int launch_permute_gamma(const ptycho_plan_s *p, const float2 *src, float2 *dst, bool to_natural,
                         cudaStream_t s);
bool supported_m(int m);
int frames_per_block(int m);
int frame_update_grid(int m, int variant, int n_items, int blocks_per_sm, int *grid, int *max_per_sm);
int frame_groups(int m, int J, int variant);
int rf_parts(int m, int J, int variant);
void fill_frame_args(const ptycho_plan_s *p, FrameArgs out[2]);
int launch_frame_update_table(int m, int variant, const FrameArgs *tab, const int2 *items, int n_items, int grid, int parity,
                              cudaStream_t s);
int prepare_kernels(int m);

// fft256_kernels.cu (m = 256): the frame update runs as the three passes over
// an L2 intermediate (launch variant 0) or as one cluster launch (variant 1)
int frame_update_256(ptycho_plan_s *p, cudaStream_t s);
int rf_parts_256(int J, int variant);
int forward_256(const ptycho_plan_s *p, const float2 *u, const float2 *w, float2 *out, cudaStream_t s);
int ifft_256(const ptycho_plan_s *p, const float2 *in, float2 *out, cudaStream_t s);
int loss_256(ptycho_plan_s *p, const float2 *u, const float2 *w, cudaStream_t s, float2 *h_out = nullptr);
int loss_256_sub(ptycho_plan_s *p, cudaStream_t s);
int probe_avg_256(ptycho_plan_s *p, cudaStream_t s);
int ingest_256(ptycho_plan_s *p, const float *f, float *part, cudaStream_t s);
int permute_256(const ptycho_plan_s *p, const float2 *src, float2 *dst, bool to_natural, cudaStream_t s);

// gather_kernels.cu
int launch_subdomain_update(ptycho_plan_s *p, cudaStream_t s);
void fill_sub_args(const ptycho_plan_s *p, SubArgs out[2]);
int launch_subdomain_update_table(bool blind, const SubArgs *tab, const int2 *items, int n_items, int parity,
                                  cudaStream_t s);
int launch_image_gather(const ptycho_plan_s *p, const float2 *q, const float2 *w, float2 *out,
                        cudaStream_t s);
// periodic plans: u (H x W) -> d_upad with u[(R mod H) (C mod W)] at (R, C);
// d_gpad -> out (H x W), out(R, C) = the sum of d_gpad over (R + a H, C + b W),
// (a, b) in {0, 1}^2 row-major, within img_rows x img_cols
// m = 256: frames per wave and chains of waves side by side (chains capped by
// the number of waves); grows the intermediate and makes streams as needed.
int configure_waves(ptycho_plan_s *p, int wave_frames, int chains, cudaStream_t s);
int launch_wrap_pad(const ptycho_plan_s *p, const float2 *u, cudaStream_t s);
int launch_fold(const ptycho_plan_s *p, float2 *out, cudaStream_t s);
int launch_probe_reduce(ptycho_plan_s *p, const float2 *u_img, float2 *grad_w, cudaStream_t s,
                        const float2 *h = nullptr);
int launch_loss_reduce(ptycho_plan_s *p, float *loss, cudaStream_t s);
int launch_metrics(ptycho_plan_s *p, cudaStream_t s);
int launch_scale(float2 *x, int64_t n, float sc, cudaStream_t s);
int launch_consensus(ptycho_plan_s *p, float *part, double *out, cudaStream_t s);
int launch_snr(ptycho_plan_s *p, const float2 *truth, const uint8_t *mask, float *part, double *out,
               cudaStream_t s);
int launch_operator_norms(ptycho_plan_s *p, uint32_t *out, cudaStream_t s);
int launch_frame_residual(ptycho_plan_s *p, const float2 *snap, float *part, double *out, cudaStream_t s);
int launch_peak_probe(int kind, int n_blocks, int iters, float *sink, cudaStream_t s);
int launch_until_init(int32_t *st, int32_t max_iter, float tol, cudaStream_t s);
int conditional_selftest(int32_t *scratch, int *ok, cudaStream_t s);
int add_until_check_node(cudaGraphNode_t *node, cudaGraph_t graph, const cudaGraphNode_t *dep, ptycho_plan_s *p,
                         cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_second, int set_second);
int launch_probe_init(ptycho_plan_s *p, float2 *w0, cudaStream_t s);
int launch_slot_rank(ptycho_plan_s *p, int32_t *setup, cudaStream_t s);
// Split m = R1 * R2 of the frame update's FFT, which fixes the task order of
// the slot ranks (m = 256: R1 = R2 = 0, natural order).
void rank_radix(int m, int *R1, int *R2);
int launch_sum_sqrtf(ptycho_plan_s *p, cudaStream_t s);
int launch_init_state(ptycho_plan_s *p, const float2 *u0, const float2 *w0, cudaStream_t s);
int launch_illumination(ptycho_plan_s *p, cudaStream_t s);
int launch_q_from_slots(const ptycho_plan_s *p, float2 *dst, cudaStream_t s);
int launch_merge(const ptycho_plan_s *p, float2 *out, cudaStream_t s);
// copy the rows of a halo message between the plan's current state and msg
int launch_halo_copy(const ptycho_plan_s *p, const HaloRow *rows, int n_rows, float2 *msg, bool pack,
                     cudaStream_t s);
int launch_prox(const float2 *y, const float *f, float2 *z, int64_t n, float eps, float lam,
                cudaStream_t s);

}  // namespace od2p
