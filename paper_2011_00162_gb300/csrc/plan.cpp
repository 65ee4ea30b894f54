// Host runtime of the OD2P library: argument checks, the overlapping domain
// decomposition, gather tile lists, plan-owned device memory, CUDA-graph
// replay of the iteration, and the extern "C" entry points of include/od2p.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "od2p_internal.h"

namespace od2p {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }
int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char *what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return PTYCHO_ERR_CUDA;
}

namespace {

// Plans and batches take their device memory from one stream-ordered pool per
// device that keeps what they free (release threshold: unlimited), so that
// creating and destroying plans of a repeated workload asks the driver for no
// new memory.  ptycho_release_cached_memory hands the cached part back.
constexpr int MAX_DEVICES = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[MAX_DEVICES] = {};

int device_pool(cudaMemPool_t *out)
{
    int dev = 0;
    OD2P_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(PTYCHO_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        OD2P_CUDA(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = ~0ull;
        OD2P_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return PTYCHO_OK;
}

// count elements of T from the pool, ordered on stream s (usable on other
// streams once s has been synchronised); recorded in `owned` for release
template <class T>
int dev_alloc(T **ptr, size_t count, std::vector<void *> &owned, cudaStream_t s)
{
    *ptr = nullptr;
    if (count == 0) count = 1;
    cudaMemPool_t pool = nullptr;
    if (int rc = device_pool(&pool)) return rc;
    cudaError_t e = cudaMallocFromPoolAsync((void **)ptr, sizeof(T) * count, pool, s);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(PTYCHO_ERR_OOM, "device allocation of " + std::to_string(sizeof(T) * count) +
                                        " bytes failed: " + cudaGetErrorString(e));
    }
    owned.push_back((void *)*ptr);
    return PTYCHO_OK;
}

// Return plan memory to the pool after the device has finished with it.
void release_owned(std::vector<void *> &owned)
{
    for (void *ptr : owned) cudaFreeAsync(ptr, nullptr);
    owned.clear();
    cudaStreamSynchronize(nullptr);
}

template <class T>
int upload(T **dst, const std::vector<T> &src, std::vector<void *> &owned, cudaStream_t s)
{
    if (int rc = dev_alloc(dst, src.size(), owned, s)) return rc;
    if (!src.empty())
        OD2P_CUDA(cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, s));
    return PTYCHO_OK;
}

// Overlapping decomposition (sections 2.1 and 3.1; rule stated in od2p.h).
// Periodic boundaries: rectangles in extended coordinates (pixel (R, C) is image
// pixel (R mod H, C mod W)), each frame at the copy of its offset whose centre
// lies on the image (`placed`), and pairs (d, e, s) over shifts s of whole
// periods, in d's coordinates, including a subdomain with copies of itself.
struct Layout {
    std::vector<int32_t> frame_sub, rect, pair, pair_rect;
    std::vector<int32_t> placed;      // J x 2: each frame's offset in extended coordinates
    std::vector<int32_t> pair_shift;  // P x 2: (s_r, s_c) in periods (0 without periodic boundaries)
};

Layout decompose(int H, int W, int m, const std::vector<int32_t> &offs, int sub_rows, int sub_cols,
                 int overlap_px, bool periodic = false)
{
    Layout L;
    const int J = (int)offs.size() / 2, D = sub_rows * sub_cols;
    std::vector<int64_t> rb(sub_rows + 1), cb(sub_cols + 1);
    for (int k = 0; k <= sub_rows; ++k) rb[k] = (int64_t)k * H / sub_rows;
    for (int k = 0; k <= sub_cols; ++k) cb[k] = (int64_t)k * W / sub_cols;
    const int grow = (overlap_px + 1) / 2;
    L.rect.resize(4 * D);
    for (int d = 0; d < D; ++d) {
        const int a = d / sub_cols, b = d % sub_cols;
        // on a torus every side of a tile faces a neighbour: grown on all sides, not clipped
        const int r0 = (int)rb[a] - (periodic || a > 0 ? grow : 0);
        const int r1 = (int)rb[a + 1] + (periodic || a + 1 < sub_rows ? grow : 0);
        const int c0 = (int)cb[b] - (periodic || b > 0 ? grow : 0);
        const int c1 = (int)cb[b + 1] + (periodic || b + 1 < sub_cols ? grow : 0);
        L.rect[4 * d + 0] = periodic ? r0 : std::max(r0, 0);
        L.rect[4 * d + 1] = periodic ? c0 : std::max(c0, 0);
        L.rect[4 * d + 2] = periodic ? r1 : std::min(r1, H);
        L.rect[4 * d + 3] = periodic ? c1 : std::min(c1, W);
    }
    // frame -> the core tile holding its window centre o + (m-1)/2, i.e. the last
    // boundary b with 2*b <= 2*o + m - 1
    L.frame_sub.resize(J);
    L.placed.resize(2 * (size_t)J);
    for (int j = 0; j < J; ++j) {
        int orow = offs[2 * j], ocol = offs[2 * j + 1];
        if (periodic) {  // the copy whose doubled centre lies in [0, 2H) x [0, 2W)
            if (2LL * orow + m - 1 >= 2LL * H) orow -= H;
            if (2LL * ocol + m - 1 >= 2LL * W) ocol -= W;
        }
        L.placed[2 * j] = orow;
        L.placed[2 * j + 1] = ocol;
        const int64_t cr = 2LL * orow + m - 1, cc = 2LL * ocol + m - 1;
        int a = 0, b = 0;
        for (int k = 1; k < sub_rows; ++k)
            if (2 * rb[k] <= cr) a = k;
        for (int k = 1; k < sub_cols; ++k)
            if (2 * cb[k] <= cc) b = k;
        const int d = a * sub_cols + b;
        L.frame_sub[j] = d;
        int32_t *R = &L.rect[4 * d];
        R[0] = std::min(R[0], orow);
        R[1] = std::min(R[1], ocol);
        R[2] = std::max(R[2], orow + m);
        R[3] = std::max(R[3], ocol + m);
    }
    const int smax = periodic ? PERIOD_SHIFTS : 0;
    for (int d = 0; d < D; ++d)
        for (int e = 0; e < D; ++e)
            for (int sr = -smax; sr <= smax; ++sr)
                for (int sc = -smax; sc <= smax; ++sc) {
                    if (d == e && sr == 0 && sc == 0) continue;
                    const int32_t *A = &L.rect[4 * d], *B = &L.rect[4 * e];
                    const int r0 = std::max(A[0], B[0] + sr * H), c0 = std::max(A[1], B[1] + sc * W);
                    const int r1 = std::min(A[2], B[2] + sr * H), c1 = std::min(A[3], B[3] + sc * W);
                    if (r0 < r1 && c0 < c1) {
                        L.pair.insert(L.pair.end(), {d, e});
                        L.pair_shift.insert(L.pair_shift.end(), {sr, sc});
                        L.pair_rect.insert(L.pair_rect.end(), {r0, c0, r1, c1});
                    }
                }
    return L;
}

// Pair k's reverse (e, d, -s) and whether k is the one listed first of the two
// (d < e, or d = e with the positive shift), which fixes the operand order of v.
void pair_links(const Layout &L, std::vector<int> &rev, std::vector<int> &first)
{
    const int P = (int)L.pair.size() / 2;
    rev.assign(P, -1);
    first.assign(P, 0);
    for (int k = 0; k < P; ++k) {
        const int d = L.pair[2 * k], e = L.pair[2 * k + 1], sr = L.pair_shift[2 * k], sc = L.pair_shift[2 * k + 1];
        for (int q = 0; q < P; ++q)
            if (L.pair[2 * q] == e && L.pair[2 * q + 1] == d && L.pair_shift[2 * q] == -sr &&
                L.pair_shift[2 * q + 1] == -sc)
                rev[k] = q;
        first[k] = d < e || (d == e && (sr > 0 || (sr == 0 && sc > 0)));
    }
}

// Tiles of TILE_H x TILE_W pixels over each region, with the frames whose
// windows meet the tile, ascending in j.
struct HostTiles {
    std::vector<Tile> tiles;
    std::vector<int32_t> ptr, reg_ptr;
    std::vector<ListEntry> list;
};

HostTiles make_tiles(int n_reg, const std::vector<int32_t> &reg_rect,
                     const std::vector<std::vector<int32_t>> &reg_frames,
                     const std::vector<int32_t> &offs, int m)
{
    HostTiles T;
    std::vector<std::vector<ListEntry>> lists;
    for (int g = 0; g < n_reg; ++g) {
        T.reg_ptr.push_back((int32_t)T.tiles.size());
        const int r0 = reg_rect[4 * g], c0 = reg_rect[4 * g + 1];
        const int h = reg_rect[4 * g + 2] - r0, w = reg_rect[4 * g + 3] - c0;
        const int nty = (h + TILE_H - 1) / TILE_H, ntx = (w + TILE_W - 1) / TILE_W;
        const size_t base = T.tiles.size();
        for (int ty = 0; ty < nty; ++ty)
            for (int tx = 0; tx < ntx; ++tx) T.tiles.push_back(Tile{g, ty * TILE_H, tx * TILE_W, 0});
        lists.resize(T.tiles.size());
        for (int j : reg_frames[g]) {
            const int lr = offs[2 * j] - r0, lc = offs[2 * j + 1] - c0;
            const int ty0 = std::max(0, lr / TILE_H), ty1 = std::min(nty - 1, (lr + m - 1) / TILE_H);
            const int tx0 = std::max(0, lc / TILE_W), tx1 = std::min(ntx - 1, (lc + m - 1) / TILE_W);
            for (int ty = ty0; ty <= ty1; ++ty)
                for (int tx = tx0; tx <= tx1; ++tx)
                    lists[base + (size_t)ty * ntx + tx].push_back(
                        ListEntry{j, ty * TILE_H - lr, tx * TILE_W - lc, 0});
        }
    }
    T.reg_ptr.push_back((int32_t)T.tiles.size());
    T.ptr.push_back(0);
    for (auto &l : lists) {
        T.list.insert(T.list.end(), l.begin(), l.end());
        T.ptr.push_back((int32_t)T.list.size());
    }
    return T;
}

int upload_tiles(GatherTiles &G, const HostTiles &T, std::vector<void *> &owned, cudaStream_t s)
{
    G.n_tiles = (int32_t)T.tiles.size();
    if (int rc = upload(&G.tiles, T.tiles, owned, s)) return rc;
    if (int rc = upload(&G.ptr, T.ptr, owned, s)) return rc;
    if (int rc = upload(&G.list, T.list, owned, s)) return rc;
    return upload(&G.reg_ptr, T.reg_ptr, owned, s);
}

int upload_groups(ProbeGroups &G, const std::vector<std::vector<int32_t>> &groups,
                  std::vector<void *> &owned, cudaStream_t s)
{
    std::vector<int32_t> frames, chunk_ptr;
    std::vector<int4> chunks;
    for (int g = 0; g < (int)groups.size(); ++g) {
        chunk_ptr.push_back((int32_t)chunks.size());
        const int b0 = (int)frames.size();
        frames.insert(frames.end(), groups[g].begin(), groups[g].end());
        for (int b = b0; b < (int)frames.size(); b += PROBE_CHUNK)
            chunks.push_back(make_int4(g, b, std::min<int>(b + PROBE_CHUNK, (int)frames.size()), 0));
    }
    chunk_ptr.push_back((int32_t)chunks.size());
    G.n_groups = (int32_t)groups.size();
    G.n_chunks = (int32_t)chunks.size();
    if (int rc = upload(&G.frames, frames, owned, s)) return rc;
    if (int rc = upload(&G.chunks, chunks, owned, s)) return rc;
    return upload(&G.chunk_ptr, chunk_ptr, owned, s);
}

int enqueue_iteration(ptycho_plan_s *p, cudaStream_t s)
{
    if (int rc = launch_frame_update(p, s)) return rc;
    if (p->blind) {
        if (int rc = launch_probe_avg(p, s)) return rc;
        if (int rc = launch_probe_reduce(p, nullptr, nullptr, s)) return rc;
        OD2P_CUDA(cudaMemcpyAsync(p->d_w, p->d_wnew, sizeof(float2) * p->MM, cudaMemcpyDeviceToDevice, s));
    }
    return launch_subdomain_update(p, s);
}

// One iteration from buffer parity `parity`, captured into *out (not instantiated).
int capture_iteration(ptycho_plan_s *p, int parity, cudaGraph_t *out)
{
    *out = nullptr;
    if (!p->cap_stream) OD2P_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    OD2P_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int saved = p->cur;
    p->cur = parity;
    int rc = enqueue_iteration(p, p->cap_stream);
    p->cur = saved;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    *out = g;
    return PTYCHO_OK;
}

// The iterate-until graph from parity `parity`: a device-side while loop whose
// body runs the iteration from `parity`, the stopping test, and -- if the test
// says go on -- the iteration from the other parity and the test again, so the
// loop stops after the exact iteration that met the test.
int build_until_graph(ptycho_plan_s *p, int parity)
{
    cudaGraph_t it[2] = {nullptr, nullptr}, G = nullptr;
    int rc = PTYCHO_OK;
    cudaError_t e = cudaSuccess;
    auto done = [&](int code) {
        for (cudaGraph_t g : {it[0], it[1], G})
            if (g) cudaGraphDestroy(g);
        return code;
    };
    if ((rc = capture_iteration(p, parity, &it[0])) || (rc = capture_iteration(p, parity ^ 1, &it[1])))
        return done(rc);
    if ((e = cudaGraphCreate(&G, 0)) != cudaSuccess) return done(cuda_fail(e, "cudaGraphCreate"));
    cudaGraphConditionalHandle h_loop, h_second;
    if ((e = cudaGraphConditionalHandleCreate(&h_loop, G, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
        return done(cuda_fail(e, "cudaGraphConditionalHandleCreate"));
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = h_loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t loop;
    if ((e = cudaGraphAddNode(&loop, G, nullptr, nullptr, 0, &wp)) != cudaSuccess)
        return done(cuda_fail(e, "cudaGraphAddNode (while)"));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    if ((e = cudaGraphConditionalHandleCreate(&h_second, body, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
        return done(cuda_fail(e, "cudaGraphConditionalHandleCreate"));
    cudaGraphNode_t first, test1;
    if ((e = cudaGraphAddChildGraphNode(&first, body, nullptr, 0, it[0])) != cudaSuccess)
        return done(cuda_fail(e, "cudaGraphAddChildGraphNode"));
    if ((rc = add_until_check_node(&test1, body, &first, p, h_loop, h_second, 1))) return done(rc);
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = h_second;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t second_if;
    if ((e = cudaGraphAddNode(&second_if, body, &test1, nullptr, 1, &ip)) != cudaSuccess)
        return done(cuda_fail(e, "cudaGraphAddNode (if)"));
    cudaGraph_t second_body = ip.conditional.phGraph_out[0];
    cudaGraphNode_t second, test2;
    if ((e = cudaGraphAddChildGraphNode(&second, second_body, nullptr, 0, it[1])) != cudaSuccess)
        return done(cuda_fail(e, "cudaGraphAddChildGraphNode"));
    if ((rc = add_until_check_node(&test2, second_body, &second, p, h_loop, h_second, 0))) return done(rc);
    if ((e = cudaGraphInstantiate(&p->until[parity], G, 0)) != cudaSuccess) {
        p->until[parity] = nullptr;
        return done(cuda_fail(e, "cudaGraphInstantiate (until)"));
    }
    return done(PTYCHO_OK);
}

int capture_graph(ptycho_plan_s *p, int parity)
{
    cudaGraph_t g = nullptr;
    if (int rc = capture_iteration(p, parity, &g)) return rc;
    cudaError_t e = cudaGraphInstantiate(&p->graph[parity], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        p->graph[parity] = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    return PTYCHO_OK;
}

void drop_graphs(cudaGraphExec_t g[2])
{
    for (int i = 0; i < 2; ++i)
        if (g[i]) {
            cudaGraphExecDestroy(g[i]);
            g[i] = nullptr;
        }
}

// Switch the frame update of p to launch shape `variant` with at most
// blocks_per_sm resident blocks per SM; drops the captured iteration graphs and
// zeroes the RF partials when the partial-sum layout changes.
int apply_launch(ptycho_plan_s *p, int variant, int blocks_per_sm, cudaStream_t s)
{
    if (p->fft_kind) {  // the 16 x 4 kernel has its own grid; the shape applies on return to kind 0
        p->k1_variant = variant;
        p->k1_blocks_per_sm = blocks_per_sm;
        return PTYCHO_OK;
    }
    if (p->M == 256) {  // variant 0: three passes; 1: one cluster launch (blocks_per_sm not used)
        const int parts = rf_parts(p->M, p->J, variant);
        if (parts != p->n_rf_parts || variant != p->k1_variant) {
            const int cap = std::max(rf_parts(p->M, p->J, 0), rf_parts(p->M, p->J, 1));
            OD2P_CUDA(cudaMemsetAsync(p->d_rf_part, 0, sizeof(float) * cap, s));
        }
        p->k1_variant = variant;
        p->k1_blocks_per_sm = 0;
        p->n_rf_parts = parts;
        drop_graphs(p->graph);
        drop_graphs(p->until);
        return PTYCHO_OK;
    }
    int grid = 0;
    if (int rc = frame_update_grid(p->M, variant, frame_groups(p->M, p->J, variant), blocks_per_sm, &grid, nullptr))
        return rc;
    const int parts = rf_parts(p->M, p->J, variant);
    if (parts != p->n_rf_parts || variant != p->k1_variant) {
        const int cap = std::max(rf_parts(p->M, p->J, 0), rf_parts(p->M, p->J, 1));
        OD2P_CUDA(cudaMemsetAsync(p->d_rf_part, 0, sizeof(float) * cap, s));
    }
    p->k1_variant = variant;
    p->k1_blocks_per_sm = blocks_per_sm;
    p->n_k1_blocks = grid;
    p->n_rf_parts = parts;
    drop_graphs(p->graph);
    drop_graphs(p->until);
    return PTYCHO_OK;
}

}  // namespace
}  // namespace od2p

namespace od2p {

int configure_waves(ptycho_plan_s *p, int wave_frames, int chains, cudaStream_t s)
{
    const int nch = std::max(1, std::min(chains, (p->J + wave_frames - 1) / wave_frames));
    const int64_t need = (int64_t)nch * wave_frames;
    if (need > p->t_cap_frames) {  // a larger intermediate; the old one stays with the plan until it is freed
        float2 *T = nullptr;
        if (int rc = dev_alloc(&T, (size_t)need * p->MM, p->owned, s)) return rc;
        p->d_T = T;
        p->t_cap_frames = need;
    }
    for (int i = 0; i < nch; ++i) {
        cudaError_t e = cudaSuccess;
        if (i > 0 && !p->wave_stream[i]) e = cudaStreamCreateWithFlags(&p->wave_stream[i], cudaStreamNonBlocking);
        if (e == cudaSuccess && nch > 1 && !p->wave_ev[i]) e = cudaEventCreateWithFlags(&p->wave_ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "wave streams");
    }
    p->wave_frames = wave_frames;
    p->t_waves = nch;
    return PTYCHO_OK;
}


int build_plan(ptycho_plan_t **out, const ptycho_geometry *g, const float *f_dev, const int32_t *owner,
               int32_t rank, ptycho_stream_t stream);

// Halo messages of a shard, one per peer and direction: for every ordered pair
// (e, d) in pair order with owner[e] = sender and owner[d] = receiver, the rows
// of u_e on Omega_e n Omega_d, then Lambda_{e,d}; blind, then W_e and Delta_e of
// every subdomain e the sender owns, e ascending.  Stored as row copies
// (array, length, offset in the array, offset in the message).
void halo_rows(const ptycho_plan_s *p, int sender, int receiver, std::vector<HaloRow> &rows, int64_t &n)
{
    rows.clear();
    n = 0;
    for (int k = 0; k < p->P; ++k) {
        const int e = p->pair[2 * k], d = p->pair[2 * k + 1];
        if (p->owner[e] != sender || p->owner[d] != receiver) continue;
        const int32_t *R = &p->rect[4 * e], *Pr = &p->pair_rect[4 * k];
        const int pitch = R[3] - R[1], cols = Pr[3] - Pr[1];
        for (int r = Pr[0]; r < Pr[2]; ++r) {
            rows.push_back(HaloRow{0, cols, p->u_off[e] + (int64_t)(r - R[0]) * pitch + (Pr[1] - R[1]), n});
            n += cols;
        }
        for (int r = 0; r < Pr[2] - Pr[0]; ++r) {
            rows.push_back(HaloRow{1, cols, p->lam_off[k] + (int64_t)r * cols, n});
            n += cols;
        }
    }
    if (p->blind)
        for (int e = 0; e < p->D; ++e)
            if (p->owner[e] == sender) {
                rows.push_back(HaloRow{2, p->MM, (int64_t)e * p->MM, n});
                n += p->MM;
                rows.push_back(HaloRow{3, p->MM, (int64_t)e * p->MM, n});
                n += p->MM;
            }
}

int build_halo_tables(ptycho_plan_s *p, cudaStream_t s)
{
    int world = 0;
    for (int d = 0; d < p->D; ++d) world = std::max(world, p->owner[d] + 1);
    p->world = world;
    p->halo.assign(world, ptycho_plan_s::Halo{});
    std::vector<HaloRow> rows;
    for (int q = 0; q < world; ++q) {
        if (q == p->rank) continue;
        ptycho_plan_s::Halo &h = p->halo[q];
        halo_rows(p, p->rank, q, rows, h.send_n);
        h.send_rows = (int32_t)rows.size();
        if (int rc = upload(&h.d_send, rows, p->owned, s)) return rc;
        halo_rows(p, q, p->rank, rows, h.recv_n);
        h.recv_rows = (int32_t)rows.size();
        if (int rc = upload(&h.d_recv, rows, p->owned, s)) return rc;
    }
    return PTYCHO_OK;
}

// Checks of a problem description shared by plans, shards and ptycho_decompose.
int check_geometry(const ptycho_geometry *g)
{
    if (!g || !g->offsets_host) return fail(PTYCHO_ERR_INVALID_ARG, "NULL geometry or offsets");
    if (!supported_m(g->m)) return fail(PTYCHO_ERR_UNSUPPORTED, "probe side m must be 16, 32, 48, 64, 80, 96, 128 or 256");
    if (g->n_frames < 1 || g->img_h < g->m || g->img_w < g->m)
        return fail(PTYCHO_ERR_INVALID_ARG, "need n_frames >= 1 and an image at least m x m");
    if (g->sub_rows < 1 || g->sub_cols < 1 || g->sub_rows > g->img_h || g->sub_cols > g->img_w ||
        g->overlap_px < 0)
        return fail(PTYCHO_ERR_INVALID_ARG, "bad subdomain grid or overlap");
    if (g->periodic != 0 && g->periodic != 1) return fail(PTYCHO_ERR_INVALID_ARG, "periodic must be 0 or 1");
    for (int j = 0; j < g->n_frames; ++j) {
        const int r0 = g->offsets_host[2 * j], c0 = g->offsets_host[2 * j + 1];
        const bool bad = g->periodic ? (r0 < 0 || c0 < 0 || r0 >= g->img_h || c0 >= g->img_w)
                                     : (r0 < 0 || c0 < 0 || r0 > g->img_h - g->m || c0 > g->img_w - g->m);
        if (bad) return fail(PTYCHO_ERR_INVALID_ARG, "offset of frame " + std::to_string(j) + " out of range");
    }
    return PTYCHO_OK;
}

// Periodic boundaries: every rectangle within (-H, 2H) x (-W, 2W), so that shifts
// of up to PERIOD_SHIFTS periods find every copy of a pixel.
int check_periodic_rects(const ptycho_geometry *g, const Layout &L)
{
    if (!g->periodic) return PTYCHO_OK;
    for (size_t d = 0; d < L.rect.size() / 4; ++d) {
        const int32_t *R = &L.rect[4 * d];
        if (R[0] <= -g->img_h || R[2] >= 2 * g->img_h || R[1] <= -g->img_w || R[3] >= 2 * g->img_w)
            return fail(PTYCHO_ERR_INVALID_ARG, "periodic: subdomain " + std::to_string(d) +
                                                    " reaches a period beyond the image (more subdomains or less overlap)");
    }
    return PTYCHO_OK;
}

}  // namespace od2p

using namespace od2p;

extern "C" {

const char *ptycho_last_error(void) { return od2p::g_err.c_str(); }

int32_t ptycho_abi_version(void) { return 3; }

int ptycho_release_cached_memory(void)
{
    cudaMemPool_t pool = nullptr;
    if (int rc = device_pool(&pool)) return rc;
    OD2P_CUDA(cudaDeviceSynchronize());
    OD2P_CUDA(cudaMemPoolTrimTo(pool, 0));
    return PTYCHO_OK;
}

int ptycho_plan(ptycho_plan_t **out, const ptycho_geometry *g, const float *f_dev,
                ptycho_stream_t stream)
{
    return build_plan(out, g, f_dev, nullptr, 0, stream);
}

int ptycho_plan_destroy(ptycho_plan_t *plan)
{
    if (!plan) return PTYCHO_OK;
    ptycho_plan_s *p = plan;
    cudaDeviceSynchronize();
    for (int i = 0; i < 2; ++i) {
        if (p->graph[i]) cudaGraphExecDestroy(p->graph[i]);
        if (p->until[i]) cudaGraphExecDestroy(p->until[i]);
    }
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    for (cudaStream_t ws : p->wave_stream)
        if (ws) cudaStreamDestroy(ws);
    for (cudaEvent_t ev : p->wave_ev)
        if (ev) cudaEventDestroy(ev);
    release_owned(p->owned);
    delete p;
    cudaGetLastError();
    return PTYCHO_OK;
}

int ptycho_decompose(const ptycho_geometry *g, int32_t *frame_sub_host, int32_t *rect_host)
{
    if (int rc = check_geometry(g)) return rc;
    std::vector<int32_t> offs(g->offsets_host, g->offsets_host + 2 * g->n_frames);
    Layout L = decompose(g->img_h, g->img_w, g->m, offs, g->sub_rows, g->sub_cols, g->overlap_px, g->periodic != 0);
    if (int rc = check_periodic_rects(g, L)) return rc;
    if (frame_sub_host) std::memcpy(frame_sub_host, L.frame_sub.data(), sizeof(int32_t) * g->n_frames);
    if (rect_host) std::memcpy(rect_host, L.rect.data(), sizeof(int32_t) * L.rect.size());
    return PTYCHO_OK;
}

int ptycho_plan_shard(ptycho_plan_t **out, const ptycho_geometry *g, const int32_t *owner_host, int32_t rank,
                      const float *f_dev, ptycho_stream_t stream)
{
    if (!out) return fail(PTYCHO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (int rc = check_geometry(g)) return rc;
    if (!owner_host) return fail(PTYCHO_ERR_INVALID_ARG, "owner is NULL");
    const int D = g->sub_rows * g->sub_cols;
    bool mine = false;
    for (int d = 0; d < D; ++d) {
        if (owner_host[d] < 0 || owner_host[d] >= D) return fail(PTYCHO_ERR_INVALID_ARG, "owner out of range");
        mine = mine || owner_host[d] == rank;
    }
    if (rank < 0 || !mine) return fail(PTYCHO_ERR_INVALID_ARG, "rank owns no subdomain");
    return build_plan(out, g, f_dev, owner_host, rank, stream);
}

int ptycho_plan_frames(const ptycho_plan_t *plan, int32_t *n_frames, int32_t *global_index_host)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    if (n_frames) *n_frames = plan->J;
    if (global_index_host) std::memcpy(global_index_host, plan->global_j.data(), sizeof(int32_t) * plan->J);
    return PTYCHO_OK;
}

static int halo_peer(const ptycho_plan_t *plan, int32_t peer)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    if (plan->owner.empty()) return fail(PTYCHO_ERR_STATE, "not a shard plan");
    if (peer < 0 || peer >= plan->world || peer == plan->rank) return fail(PTYCHO_ERR_INVALID_ARG, "bad peer rank");
    return PTYCHO_OK;
}

int od2p_halo_size(const ptycho_plan_t *plan, int32_t peer, int64_t *send_elems, int64_t *recv_elems)
{
    if (int rc = halo_peer(plan, peer)) return rc;
    if (send_elems) *send_elems = plan->halo[peer].send_n;
    if (recv_elems) *recv_elems = plan->halo[peer].recv_n;
    return PTYCHO_OK;
}

int od2p_halo_pack(const ptycho_plan_t *plan, int32_t peer, ptycho_c32 *send_dev, ptycho_stream_t stream)
{
    if (int rc = halo_peer(plan, peer)) return rc;
    const auto &h = plan->halo[peer];
    if (h.send_n && !send_dev) return fail(PTYCHO_ERR_INVALID_ARG, "send buffer is NULL");
    return launch_halo_copy(plan, h.d_send, h.send_rows, reinterpret_cast<float2 *>(send_dev), true,
                            reinterpret_cast<cudaStream_t>(stream));
}

int od2p_halo_unpack(ptycho_plan_t *plan, int32_t peer, const ptycho_c32 *recv_dev, ptycho_stream_t stream)
{
    if (int rc = halo_peer(plan, peer)) return rc;
    const auto &h = plan->halo[peer];
    if (h.recv_n && !recv_dev) return fail(PTYCHO_ERR_INVALID_ARG, "receive buffer is NULL");
    return launch_halo_copy(plan, h.d_recv, h.recv_rows, const_cast<float2 *>(reinterpret_cast<const float2 *>(recv_dev)),
                            false, reinterpret_cast<cudaStream_t>(stream));
}

int ptycho_plan_dims(const ptycho_plan_t *plan, int32_t *n_sub, int32_t *n_pairs, int64_t *u_len,
                     int64_t *lambda_len)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    if (n_sub) *n_sub = plan->D;
    if (n_pairs) *n_pairs = plan->P;
    if (u_len) *u_len = plan->u_len;
    if (lambda_len) *lambda_len = plan->lam_len;
    return PTYCHO_OK;
}

int ptycho_plan_layout(const ptycho_plan_t *plan, int32_t *frame_sub, int32_t *rect, int32_t *pair,
                       int32_t *pair_rect)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    if (frame_sub) std::memcpy(frame_sub, plan->frame_sub.data(), sizeof(int32_t) * plan->J);
    if (rect) std::memcpy(rect, plan->rect.data(), sizeof(int32_t) * 4 * plan->D);
    if (pair && plan->P) std::memcpy(pair, plan->pair.data(), sizeof(int32_t) * 2 * plan->P);
    if (pair_rect && plan->P) std::memcpy(pair_rect, plan->pair_rect.data(), sizeof(int32_t) * 4 * plan->P);
    return PTYCHO_OK;
}

int ptycho_plan_periodic_layout(const ptycho_plan_t *plan, int32_t *pair_shift, int32_t *placed)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    if (pair_shift && plan->P) std::memcpy(pair_shift, plan->pair_shift.data(), sizeof(int32_t) * 2 * plan->P);
    if (placed) std::memcpy(placed, plan->offs.data(), sizeof(int32_t) * 2 * plan->J);
    return PTYCHO_OK;
}

// The image whose windows the image-space operators read: u itself, or for a
// periodic plan its wrapped copy (no window wraps there).
static const float2 *window_source(const ptycho_plan_t *plan, const float2 *u, cudaStream_t s, int *rc)
{
    *rc = PTYCHO_OK;
    if (!plan->periodic) return u;
    *rc = launch_wrap_pad(plan, u, s);
    return plan->d_upad;
}

// A^*-type sums of frames h into the image: straight into out, or for a periodic
// plan into the padded grid and then folded onto the image.
static int gather_image(const ptycho_plan_t *plan, const float2 *h, const float2 *w, float2 *out, cudaStream_t s)
{
    if (!plan->periodic) return launch_image_gather(plan, h, w, out, s);
    if (int rc = launch_image_gather(plan, h, w, plan->d_gpad, s)) return rc;
    return launch_fold(plan, out, s);
}

int ptycho_forward(const ptycho_plan_t *plan, const ptycho_c32 *u, const ptycho_c32 *w,
                   ptycho_c32 *frames_out, ptycho_stream_t stream)
{
    if (!plan || !u || !w || !frames_out) return fail(PTYCHO_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int rc = PTYCHO_OK;
    const float2 *src = window_source(plan, reinterpret_cast<const float2 *>(u), s, &rc);
    if (rc) return rc;
    return launch_forward(plan, src, reinterpret_cast<const float2 *>(w), reinterpret_cast<float2 *>(frames_out), s);
}

int stagm_prox(const ptycho_c32 *y, const float *f, ptycho_c32 *z, int64_t n, float eps, float lambda,
               ptycho_stream_t stream)
{
    if (n < 0) return fail(PTYCHO_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!y || !f || !z)) return fail(PTYCHO_ERR_INVALID_ARG, "NULL argument");
    if (!(eps > 0.f && eps < 1.f) || !(lambda > 0.f))
        return fail(PTYCHO_ERR_INVALID_ARG, "need 0 < eps < 1 and lambda > 0");
    if (n == 0) return PTYCHO_OK;
    return launch_prox(reinterpret_cast<const float2 *>(y), f, reinterpret_cast<float2 *>(z), n, eps,
                       lambda, reinterpret_cast<cudaStream_t>(stream));
}

int overlap_add(ptycho_plan_t *plan, const ptycho_c32 *frames, const ptycho_c32 *w, ptycho_c32 *image_out,
                int32_t flags, ptycho_stream_t stream)
{
    if (!plan || !frames || !w || !image_out) return fail(PTYCHO_ERR_INVALID_ARG, "NULL argument");
    if (flags & ~PTYCHO_OA_IFFT) return fail(PTYCHO_ERR_INVALID_ARG, "unknown flag");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float2 *fr = reinterpret_cast<const float2 *>(frames);
    const float2 *wv = reinterpret_cast<const float2 *>(w);
    if (flags & PTYCHO_OA_IFFT) {
        if (int rc = launch_frames_ifft_weight(plan, fr, nullptr, true, plan->d_q, s)) return rc;
        fr = plan->d_q;
    }
    return gather_image(plan, fr, wv, reinterpret_cast<float2 *>(image_out), s);
}

int od2p_init(ptycho_plan_t *plan, const ptycho_c32 *u0, const ptycho_c32 *w0, ptycho_stream_t stream)
{
    if (!plan || !w0) return fail(PTYCHO_ERR_INVALID_ARG, "NULL plan or probe");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (int rc = launch_init_state(plan, reinterpret_cast<const float2 *>(u0), reinterpret_cast<const float2 *>(w0), s))
        return rc;
    OD2P_CUDA(cudaMemsetAsync(plan->d_gamma, 0, sizeof(float2) * (size_t)plan->J * plan->MM, s));
    OD2P_CUDA(cudaMemsetAsync(plan->d_lam[0], 0, sizeof(float2) * std::max<int64_t>(plan->lam_len, 1), s));
    OD2P_CUDA(cudaMemsetAsync(plan->d_lam[1], 0, sizeof(float2) * std::max<int64_t>(plan->lam_len, 1), s));
    if (plan->blind) OD2P_CUDA(cudaMemsetAsync(plan->d_Delta, 0, sizeof(float2) * (size_t)plan->D * plan->MM, s));
    else if (int rc = launch_illumination(plan, s)) return rc;  // the known probe's A_d^*A_d
    plan->initialised = true;
    return PTYCHO_OK;
}

int od2p_frame_update(ptycho_plan_t *plan, ptycho_stream_t stream)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    if (!plan->initialised) return fail(PTYCHO_ERR_STATE, "od2p_init has not been called");
    return launch_frame_update(plan, reinterpret_cast<cudaStream_t>(stream));
}

int probe_update(ptycho_plan_t *plan, ptycho_stream_t stream)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    if (!plan->blind) return fail(PTYCHO_ERR_STATE, "probe_update needs a blind plan");
    if (!plan->initialised) return fail(PTYCHO_ERR_STATE, "od2p_init has not been called");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (int rc = launch_probe_avg(plan, s)) return rc;
    if (int rc = launch_probe_reduce(plan, nullptr, nullptr, s)) return rc;
    OD2P_CUDA(cudaMemcpyAsync(plan->d_w, plan->d_wnew, sizeof(float2) * plan->MM, cudaMemcpyDeviceToDevice, s));
    return PTYCHO_OK;
}

int od2p_subdomain_update(ptycho_plan_t *plan, ptycho_stream_t stream)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    if (!plan->initialised) return fail(PTYCHO_ERR_STATE, "od2p_init has not been called");
    if (int rc = launch_subdomain_update(plan, reinterpret_cast<cudaStream_t>(stream))) return rc;
    plan->cur ^= 1;
    return PTYCHO_OK;
}

int od2p_iterate(ptycho_plan_t *plan, int32_t n_iter, ptycho_stream_t stream)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    if (n_iter < 0) return fail(PTYCHO_ERR_INVALID_ARG, "n_iter < 0");
    if (!plan->initialised) return fail(PTYCHO_ERR_STATE, "od2p_init has not been called");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (int i = 0; i < n_iter; ++i) {
        if (!plan->graph[plan->cur])
            if (int rc = capture_graph(plan, plan->cur)) return rc;
        OD2P_CUDA(cudaGraphLaunch(plan->graph[plan->cur], s));
        plan->cur ^= 1;
    }
    return PTYCHO_OK;
}

int od2p_iterate_until(ptycho_plan_t *plan, float rf_tol, int32_t max_iter, int32_t *n_done_host,
                       float *rf_host, ptycho_stream_t stream)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    if (max_iter < 0 || !std::isfinite(rf_tol)) return fail(PTYCHO_ERR_INVALID_ARG, "need max_iter >= 0, finite tol");
    if (!plan->initialised) return fail(PTYCHO_ERR_STATE, "od2p_init has not been called");
    if (plan->batch_member) return fail(PTYCHO_ERR_STATE, "a batch member iterates with its batch");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int32_t h[4] = {0, max_iter, 0, 0};
    if (max_iter > 0) {
        if (!plan->until[plan->cur]) {
            // the loop ends only through a device-set condition: check once per
            // plan that such a condition takes effect (a graph with no loop)
            if (!plan->cond_checked) {
                int ok = 0;
                if (int rc = conditional_selftest(plan->d_until, &ok, s)) return rc;
                if (!ok) return fail(PTYCHO_ERR_UNSUPPORTED, "device-set graph conditions have no effect here");
                plan->cond_checked = true;
            }
            if (int rc = build_until_graph(plan, plan->cur)) return rc;
        }
        if (int rc = launch_until_init(plan->d_until, max_iter, rf_tol, s)) return rc;
        OD2P_CUDA(cudaGraphLaunch(plan->until[plan->cur], s));
        OD2P_CUDA(cudaMemcpyAsync(h, plan->d_until, sizeof(h), cudaMemcpyDeviceToHost, s));
        OD2P_CUDA(cudaStreamSynchronize(s));
        if (h[0] < 1 || h[0] > max_iter) return fail(PTYCHO_ERR_CUDA, "iterate-until loop count out of range");
        plan->cur ^= (h[0] & 1);
    }
    if (n_done_host) *n_done_host = h[0];
    if (rf_host) std::memcpy(rf_host, &h[3], sizeof(float));
    return PTYCHO_OK;
}

int od2p_merge(const ptycho_plan_t *plan, ptycho_c32 *u_out, ptycho_stream_t stream)
{
    if (!plan || !u_out) return fail(PTYCHO_ERR_INVALID_ARG, "NULL argument");
    return launch_merge(plan, reinterpret_cast<float2 *>(u_out), reinterpret_cast<cudaStream_t>(stream));
}

int od2p_metrics(ptycho_plan_t *plan, float *rf, float *re, float *loss, ptycho_stream_t stream)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    if (loss && !plan->initialised) return fail(PTYCHO_ERR_STATE, "the loss needs od2p_init first");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (int rc = launch_metrics(plan, s)) return rc;
    float *d_loss = reinterpret_cast<float *>(plan->d_metrics + 4);
    if (loss) {
        if (int rc = launch_metrics_loss(plan, s)) return rc;
        if (int rc = launch_loss_reduce(plan, d_loss, s)) return rc;
    }
    double h[2];
    float hl = 0.f;
    int32_t err = 0;
    OD2P_CUDA(cudaMemcpyAsync(h, plan->d_metrics, sizeof(h), cudaMemcpyDeviceToHost, s));
    if (loss) OD2P_CUDA(cudaMemcpyAsync(&hl, d_loss, sizeof(hl), cudaMemcpyDeviceToHost, s));
    OD2P_CUDA(cudaMemcpyAsync(&err, plan->d_err, sizeof(err), cudaMemcpyDeviceToHost, s));
    OD2P_CUDA(cudaStreamSynchronize(s));
    if (err) return fail(PTYCHO_ERR_TIMEOUT, "a frame-update pipeline wait gave up (device error flag set)");
    if (rf) *rf = (float)h[0];
    if (re) *re = (float)h[1];
    if (loss) *loss = hl;
    return PTYCHO_OK;
}

int od2p_set_penalties(ptycho_plan_t *plan, float eta, float r, ptycho_stream_t stream)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    if (!(eta > 0.f) || !(r >= 0.f) || !std::isfinite(eta) || !std::isfinite(r))
        return fail(PTYCHO_ERR_INVALID_ARG, "need eta > 0 and r >= 0");
    if (plan->batch_member) return fail(PTYCHO_ERR_STATE, "the penalties of a batch member are fixed");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ptycho_plan_s *p = plan;
    // keep the unscaled multipliers eta Gamma and r Lambda
    if (eta != p->eta)
        if (int rc = launch_scale(p->d_gamma, (int64_t)p->J * p->MM, p->eta / eta, s)) return rc;
    if (r > 0.f && r != p->r)
        if (int rc = launch_scale(p->d_lam[p->cur], p->lam_len, p->r / r, s)) return rc;
    p->eta = eta;
    p->r = r;
    fill_frame_args(p, p->h_fargs);
    fill_sub_args(p, p->h_sargs);
    OD2P_CUDA(cudaMemcpyAsync(p->d_fargs, p->h_fargs, sizeof(p->h_fargs), cudaMemcpyHostToDevice, s));
    OD2P_CUDA(cudaMemcpyAsync(p->d_sargs, p->h_sargs, sizeof(p->h_sargs), cudaMemcpyHostToDevice, s));
    OD2P_CUDA(cudaStreamSynchronize(s));  // the host argument copies are read by the next launches
    drop_graphs(p->graph);
    drop_graphs(p->until);
    return PTYCHO_OK;
}

int od2p_consensus_residual(ptycho_plan_t *plan, float *rc_host, ptycho_stream_t stream)
{
    if (!plan || !rc_host) return fail(PTYCHO_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (int rc = launch_consensus(plan, plan->d_rc_part, plan->d_metrics + 3, s)) return rc;
    double h = 0.0;
    OD2P_CUDA(cudaMemcpyAsync(&h, plan->d_metrics + 3, sizeof(h), cudaMemcpyDeviceToHost, s));
    OD2P_CUDA(cudaStreamSynchronize(s));
    *rc_host = (float)h;
    return PTYCHO_OK;
}

int ptycho_peak_probe(int32_t kind, int32_t n_blocks, int32_t iters, float *sink_dev, ptycho_stream_t stream)
{
    if ((kind != PTYCHO_PROBE_FMA && kind != PTYCHO_PROBE_SMEM) || n_blocks <= 0 || iters <= 0 || !sink_dev)
        return fail(PTYCHO_ERR_INVALID_ARG, "need kind 0 or 1, n_blocks > 0, iters > 0 and a sink");
    return launch_peak_probe(kind, n_blocks, iters, sink_dev, reinterpret_cast<cudaStream_t>(stream));
}

int od2p_gamma_snapshot(ptycho_plan_t *plan, ptycho_stream_t stream)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t n = (size_t)plan->J * plan->MM;
    if (!plan->d_gamma_snap)
        if (int rc = dev_alloc(&plan->d_gamma_snap, n, plan->owned, s)) return rc;
    OD2P_CUDA(cudaMemcpyAsync(plan->d_gamma_snap, plan->d_gamma, sizeof(float2) * n, cudaMemcpyDeviceToDevice, s));
    return PTYCHO_OK;
}

int od2p_frame_residual(ptycho_plan_t *plan, float *res_host, ptycho_stream_t stream)
{
    if (!plan || !res_host) return fail(PTYCHO_ERR_INVALID_ARG, "NULL argument");
    if (!plan->d_gamma_snap) return fail(PTYCHO_ERR_STATE, "od2p_gamma_snapshot has not been called");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (int rc = launch_frame_residual(plan, plan->d_gamma_snap, plan->d_snr_part, plan->d_snr, s)) return rc;
    double h = 0.0;
    OD2P_CUDA(cudaMemcpyAsync(&h, plan->d_snr, sizeof(h), cudaMemcpyDeviceToHost, s));
    OD2P_CUDA(cudaStreamSynchronize(s));
    *res_host = (float)h;
    return PTYCHO_OK;
}

int od2p_operator_norms(ptycho_plan_t *plan, float *norms_host, ptycho_stream_t stream)
{
    if (!plan || !norms_host) return fail(PTYCHO_ERR_INVALID_ARG, "NULL argument");
    if (plan->blind) return fail(PTYCHO_ERR_STATE, "operator norms need a nonblind plan (a known probe)");
    if (!plan->initialised) return fail(PTYCHO_ERR_STATE, "od2p_init has not been called");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (int rc = launch_operator_norms(plan, plan->d_opn, s)) return rc;
    uint32_t h[2] = {0u, 0u};
    OD2P_CUDA(cudaMemcpyAsync(h, plan->d_opn, sizeof(h), cudaMemcpyDeviceToHost, s));
    OD2P_CUDA(cudaStreamSynchronize(s));
    std::memcpy(norms_host, h, sizeof(h));  // non-negative floats kept as their bit patterns
    return PTYCHO_OK;
}

int od2p_snr(ptycho_plan_t *plan, const ptycho_c32 *truth_dev, const uint8_t *mask_dev, float *snr_host,
             ptycho_stream_t stream)
{
    if (!plan || !truth_dev || !snr_host) return fail(PTYCHO_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (int rc = launch_snr(plan, reinterpret_cast<const float2 *>(truth_dev), mask_dev, plan->d_snr_part,
                            plan->d_snr, s))
        return rc;
    double h = 0.0;
    OD2P_CUDA(cudaMemcpyAsync(&h, plan->d_snr + 2, sizeof(h), cudaMemcpyDeviceToHost, s));
    OD2P_CUDA(cudaStreamSynchronize(s));
    *snr_host = (float)h;
    return PTYCHO_OK;
}

int ptycho_probe_init(ptycho_plan_t *plan, ptycho_c32 *w0_dev, ptycho_stream_t stream)
{
    if (!plan || !w0_dev) return fail(PTYCHO_ERR_INVALID_ARG, "NULL argument");
    return launch_probe_init(plan, reinterpret_cast<float2 *>(w0_dev), reinterpret_cast<cudaStream_t>(stream));
}

static int set_fft_kind(ptycho_plan_t *plan, int32_t kind, cudaStream_t s);

int ptycho_plan_set_fft(ptycho_plan_t *plan, int32_t kind, ptycho_stream_t stream)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    if (kind < 0 || kind > 2) return fail(PTYCHO_ERR_INVALID_ARG, "fft kind must be 0, 1 or 2");
    if (kind && plan->M != 64) return fail(PTYCHO_ERR_UNSUPPORTED, "fft kinds 1 and 2 are for m = 64");
    if (plan->batch_member) return fail(PTYCHO_ERR_STATE, "a batch member runs its batch's frame update");
    return set_fft_kind(plan, kind, reinterpret_cast<cudaStream_t>(stream));
}

static int set_fft_kind(ptycho_plan_t *plan, int32_t kind, cudaStream_t s)
{
    if (kind == plan->fft_kind) return PTYCHO_OK;
    if (kind == 0) {
        plan->fft_kind = 0;
        plan->n_rf_parts = -1;  // forces the partials to be cleared
        return apply_launch(plan, plan->k1_variant, plan->k1_blocks_per_sm, s);
    }
    int grid = 0;
    if (int rc = f4_grid(kind, plan->J, &grid)) return rc;
    const int cap = std::max(rf_parts(plan->M, plan->J, 0), rf_parts(plan->M, plan->J, 1));
    OD2P_CUDA(cudaMemsetAsync(plan->d_rf_part, 0, sizeof(float) * cap, s));
    plan->fft_kind = kind;
    plan->n_k1_blocks = grid;
    plan->n_rf_parts = plan->J * (256 / 32);
    drop_graphs(plan->graph);
    drop_graphs(plan->until);
    return PTYCHO_OK;
}

int ptycho_plan_get_fft(const ptycho_plan_t *plan, int32_t *kind)
{
    if (!plan || !kind) return fail(PTYCHO_ERR_INVALID_ARG, "NULL argument");
    *kind = plan->fft_kind;
    return PTYCHO_OK;
}

int ptycho_plan_set_launch(ptycho_plan_t *plan, int32_t variant, int32_t blocks_per_sm, ptycho_stream_t stream)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    if (variant < 0 || variant >= PTYCHO_LAUNCH_VARIANTS) return fail(PTYCHO_ERR_INVALID_ARG, "variant out of range");
    if (blocks_per_sm < 0) return fail(PTYCHO_ERR_INVALID_ARG, "blocks_per_sm < 0");
    if (plan->batch_member)
        return fail(PTYCHO_ERR_STATE, "a batch member takes its launch shape from ptycho_batch_set_launch");
    return apply_launch(plan, variant, blocks_per_sm, reinterpret_cast<cudaStream_t>(stream));
}

int ptycho_plan_get_launch(const ptycho_plan_t *plan, int32_t *variant, int32_t *blocks_per_sm,
                           int32_t *max_blocks_per_sm)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    int most = 1;
    if (plan->M != 256) {
        int grid = 0;
        if (int rc = frame_update_grid(plan->M, plan->k1_variant, 1, 0, &grid, &most)) return rc;
    }
    if (variant) *variant = plan->k1_variant;
    if (blocks_per_sm) *blocks_per_sm = plan->k1_blocks_per_sm;
    if (max_blocks_per_sm) *max_blocks_per_sm = most;
    return PTYCHO_OK;
}

int ptycho_plan_get_waves(const ptycho_plan_t *plan, int32_t *wave_frames, int32_t *chains, int32_t *launches)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    const bool waves = plan->M == 256 && plan->k1_variant == 0;
    if (wave_frames) *wave_frames = waves ? plan->wave_frames : 0;
    if (chains) *chains = waves ? plan->t_waves : 1;
    if (launches) *launches = waves ? 3 * ((plan->J + plan->wave_frames - 1) / plan->wave_frames) : 1;
    return PTYCHO_OK;
}

int ptycho_plan_set_waves(ptycho_plan_t *plan, int32_t wave_frames, int32_t chains, ptycho_stream_t stream)
{
    if (!plan) return fail(PTYCHO_ERR_INVALID_ARG, "plan is NULL");
    if (plan->M != 256) return fail(PTYCHO_ERR_UNSUPPORTED, "wave shapes exist for m = 256 only");
    if (wave_frames < 1 || wave_frames > MAX_WAVE_FRAMES || chains < 1 || chains > MAX_WAVE_CHAINS)
        return fail(PTYCHO_ERR_INVALID_ARG, "need 1 <= wave_frames <= 152 and 1 <= chains <= 8");
    if (int rc = configure_waves(plan, wave_frames, chains, reinterpret_cast<cudaStream_t>(stream))) return rc;
    drop_graphs(plan->graph);
    drop_graphs(plan->until);
    return PTYCHO_OK;
}

int od2p_state_len(const ptycho_plan_t *plan, int32_t which, int64_t *n)
{
    if (!plan || !n) return fail(PTYCHO_ERR_INVALID_ARG, "NULL argument");
    switch (which) {
    case PTYCHO_STATE_U: *n = plan->u_len; break;
    case PTYCHO_STATE_GAMMA:
    case PTYCHO_STATE_Q: *n = (int64_t)plan->J * plan->MM; break;
    case PTYCHO_STATE_LAMBDA: *n = plan->lam_len; break;
    case PTYCHO_STATE_WD:
    case PTYCHO_STATE_DELTA:
        if (!plan->blind) return fail(PTYCHO_ERR_STATE, "W_d and Delta exist in blind plans only");
        *n = (int64_t)plan->D * plan->MM;
        break;
    case PTYCHO_STATE_W: *n = plan->MM; break;
    default: return fail(PTYCHO_ERR_INVALID_ARG, "unknown state selector");
    }
    return PTYCHO_OK;
}

static float2 *state_ptr(const ptycho_plan_t *p, int which)
{
    switch (which) {
    case PTYCHO_STATE_U: return p->d_u[p->cur];
    case PTYCHO_STATE_GAMMA: return p->d_gamma;
    case PTYCHO_STATE_LAMBDA: return p->d_lam[p->cur];
    case PTYCHO_STATE_WD: return p->d_Wd;
    case PTYCHO_STATE_DELTA: return p->d_Delta;
    case PTYCHO_STATE_W: return p->d_w;
    case PTYCHO_STATE_Q: return p->d_q;
    default: return nullptr;
    }
}

int od2p_get_state(const ptycho_plan_t *plan, int32_t which, ptycho_c32 *dst, ptycho_stream_t stream)
{
    int64_t n = 0;
    if (int rc = od2p_state_len(plan, which, &n)) return rc;
    if (n == 0) return PTYCHO_OK;
    if (!dst) return fail(PTYCHO_ERR_INVALID_ARG, "dst is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (which == PTYCHO_STATE_GAMMA)
        return launch_permute_gamma(plan, plan->d_gamma, reinterpret_cast<float2 *>(dst), true, s);
    if (which == PTYCHO_STATE_Q && !plan->blind) return launch_q_from_slots(plan, reinterpret_cast<float2 *>(dst), s);
    if (n) OD2P_CUDA(cudaMemcpyAsync(dst, state_ptr(plan, which), sizeof(float2) * n, cudaMemcpyDeviceToDevice, s));
    return PTYCHO_OK;
}

int od2p_set_state(ptycho_plan_t *plan, int32_t which, const ptycho_c32 *src, ptycho_stream_t stream)
{
    int64_t n = 0;
    if (int rc = od2p_state_len(plan, which, &n)) return rc;
    if (which == PTYCHO_STATE_Q) return fail(PTYCHO_ERR_INVALID_ARG, "PTYCHO_STATE_Q is read-only");
    if (n == 0) return PTYCHO_OK;
    if (!src) return fail(PTYCHO_ERR_INVALID_ARG, "src is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (which == PTYCHO_STATE_GAMMA)
        return launch_permute_gamma(plan, reinterpret_cast<const float2 *>(src), plan->d_gamma, false, s);
    if (n) OD2P_CUDA(cudaMemcpyAsync(state_ptr(plan, which), src, sizeof(float2) * n, cudaMemcpyDeviceToDevice, s));
    // a new known probe changes the nonblind denominators sum_j S_j^T |w|^2
    if (which == PTYCHO_STATE_W && !plan->blind && plan->initialised) return launch_illumination(plan, s);
    return PTYCHO_OK;
}

int stagm_loss_grad(ptycho_plan_t *plan, const ptycho_c32 *u, const ptycho_c32 *w, float *loss,
                    ptycho_c32 *grad_u, ptycho_c32 *grad_w, int32_t recompute, ptycho_stream_t stream)
{
    if (!plan || !u || !w || !loss) return fail(PTYCHO_ERR_INVALID_ARG, "NULL argument");
    if (recompute < 0 || recompute > 2) return fail(PTYCHO_ERR_INVALID_ARG, "recompute must be 0, 1 or 2");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float2 *ww = reinterpret_cast<const float2 *>(w);
    int rc0 = PTYCHO_OK;
    const float2 *uu = (recompute != 2 || grad_w) ? window_source(plan, reinterpret_cast<const float2 *>(u), s, &rc0)
                                                  : reinterpret_cast<const float2 *>(u);
    if (rc0) return rc0;
    const float2 *h = plan->d_q;
    if (recompute == 2) {  // the gradient frames stored by the last recompute = 0 call
        if (!plan->h_stored || plan->h_u != u || plan->h_w != w)
            return fail(PTYCHO_ERR_STATE, "no stored gradient frames for this u and w (call with recompute = 0 first)");
        h = plan->d_hstore;
        OD2P_CUDA(cudaMemcpyAsync(loss, plan->d_hloss, sizeof(float), cudaMemcpyDeviceToDevice, s));
    } else {
        if (recompute == 0) {
            if (!plan->d_hstore) {
                if (int rc = dev_alloc(&plan->d_hstore, (size_t)plan->J * plan->MM, plan->owned, s)) return rc;
                if (int rc = dev_alloc(&plan->d_hloss, 1, plan->owned, s)) return rc;
            }
            h = plan->d_hstore;
            plan->h_stored = false;
        }
        if (int rc = launch_loss_frames(plan, uu, ww, s, const_cast<float2 *>(h))) return rc;
        if (int rc = launch_loss_reduce(plan, loss, s)) return rc;
        if (recompute == 0) {
            OD2P_CUDA(cudaMemcpyAsync(plan->d_hloss, loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
            plan->h_stored = true;
            plan->h_u = u;
            plan->h_w = w;
        }
    }
    if (grad_u)
        if (int rc = gather_image(plan, h, ww, reinterpret_cast<float2 *>(grad_u), s)) return rc;
    if (grad_w)
        if (int rc = launch_probe_reduce(plan, uu, reinterpret_cast<float2 *>(grad_w), s, h)) return rc;
    return PTYCHO_OK;
}

// ---------------------------------------------------------------- batches
struct ptycho_batch_s {
    std::vector<ptycho_plan_s *> plans;
    struct Cls {  // the member plans of one probe side m
        int m = 0, grid = 0;
        bool f4 = false;                 // m = 64: the 16 x 4 split, one frame per item
        std::vector<ptycho_plan_s *> waves;  // m = 256: members whose own wave passes run in turn
        int n_items[2] = {0, 0};         // (plan, frame group) items per launch shape
        od2p::FrameArgs *tab = nullptr;
        int2 *items[2] = {nullptr, nullptr};
    };
    int variant = 0, blocks_per_sm = 0;
    std::vector<Cls> cls;
    od2p::SubArgs *stab = nullptr;
    int2 *titems = nullptr;        // tiles of the members that gather through slots
    int n_titems = 0;
    int2 *litems = nullptr;        // tiles of the members that gather through frame lists (blind)
    int n_litems = 0;
    std::vector<void *> owned;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int cur = 0;
    // side streams and events of the per-class branches (graph capture only)
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> side_done;
    cudaEvent_t fork = nullptr;
};

int ptycho_batch_destroy(ptycho_batch_t *b)
{
    if (!b) return PTYCHO_OK;
    cudaDeviceSynchronize();
    for (int i = 0; i < 2; ++i)
        if (b->graph[i]) cudaGraphExecDestroy(b->graph[i]);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (cudaStream_t t : b->side) cudaStreamDestroy(t);
    for (cudaEvent_t e : b->side_done) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    release_owned(b->owned);
    for (ptycho_plan_s *p : b->plans) ptycho_plan_destroy(p);
    delete b;
    cudaGetLastError();
    return PTYCHO_OK;
}

int ptycho_batch_plan(ptycho_batch_t **out, const ptycho_geometry *geoms, const float *const *f_devs, int32_t n,
                      ptycho_stream_t stream)
{
    if (!out) return fail(PTYCHO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!geoms || !f_devs || n < 1) return fail(PTYCHO_ERR_INVALID_ARG, "need n >= 1 geometries and intensity stacks");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    auto *b = new (std::nothrow) ptycho_batch_s();
    if (!b) return fail(PTYCHO_ERR_OOM, "host allocation failed");
    auto bail = [&](int rc) {
        std::string msg = od2p::g_err;
        ptycho_batch_destroy(b);
        od2p::g_err = msg;
        return rc;
    };
    for (int i = 0; i < n; ++i) {
        ptycho_plan_t *p = nullptr;
        if (int rc = ptycho_plan(&p, &geoms[i], f_devs[i], stream)) return bail(rc);
        b->plans.push_back(p);
    }
    // one table per probe side: the member plans' frame-update arguments and the
    // (plan, frame group) work items
    std::vector<int> ms;
    for (auto *p : b->plans)
        if (std::find(ms.begin(), ms.end(), p->M) == ms.end()) ms.push_back(p->M);
    std::sort(ms.begin(), ms.end());
    // m = 64 members take the 16 x 4 transform split (fft kind 2), alone and in the batch
    for (auto *p : b->plans)
        if (p->M == 64)
            if (int rc = set_fft_kind(p, 2, s)) return bail(rc);
    for (auto *p : b->plans) p->batch_member = true;
    for (int m : ms) {
        if (m == 256) {  // a 256 x 256 frame spans 16 blocks: each member runs its own waves
            ptycho_batch_s::Cls c;
            c.m = m;
            for (auto *p : b->plans)
                if (p->M == m) c.waves.push_back(p);
            b->cls.push_back(c);
            continue;
        }
        std::vector<FrameArgs> tab;
        std::vector<int2> items[2];
        const bool f4 = m == 64;
        for (auto *p : b->plans) {
            if (p->M != m) continue;
            const int local = (int)tab.size() / 2;
            tab.push_back(p->h_fargs[0]);
            tab.push_back(p->h_fargs[1]);
            for (int v = 0; v < 2; ++v) {
                const int n_it = f4 ? p->J : frame_groups(m, p->J, v);  // f4: one frame per item
                for (int g = 0; g < n_it; ++g) items[v].push_back(make_int2(local, g));
            }
        }
        ptycho_batch_s::Cls c;
        c.m = m;
        c.f4 = f4;
        c.n_items[0] = (int)items[0].size();
        c.n_items[1] = (int)items[1].size();
        int rc;
        if ((rc = upload(&c.tab, tab, b->owned, s)) || (rc = upload(&c.items[0], items[0], b->owned, s)) ||
            (rc = upload(&c.items[1], items[1], b->owned, s)) ||
            (rc = f4 ? f4_grid(2, c.n_items[0], &c.grid) : frame_update_grid(m, 0, c.n_items[0], 0, &c.grid, nullptr)))
            return bail(rc);
        b->cls.push_back(c);
    }
    // every subdomain tile of every plan for the single subdomain-update launch
    // (slot gathers and frame-list gathers -- blind members, or more than 255
    // frames over a pixel -- are two launches of the same kernel template)
    std::vector<SubArgs> stab;
    std::vector<int2> titems, litems;
    for (int i = 0; i < n; ++i) {
        stab.push_back(b->plans[i]->h_sargs[0]);
        stab.push_back(b->plans[i]->h_sargs[1]);
        const bool list = b->plans[i]->blind || !b->plans[i]->slots;
        for (int t = 0; t < b->plans[i]->sub_tiles.n_tiles; ++t) (list ? litems : titems).push_back(make_int2(i, t));
    }
    b->n_titems = (int)titems.size();
    b->n_litems = (int)litems.size();
    // streams and events for the per-class branches of the iteration graph
    for (size_t k = 1; k < b->cls.size(); ++k) {
        cudaStream_t t = nullptr;
        cudaEvent_t ev = nullptr;
        cudaError_t e1 = cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking);
        if (e1 != cudaSuccess) return bail(cuda_fail(e1, "cudaStreamCreateWithFlags"));
        b->side.push_back(t);
        if ((e1 = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return bail(cuda_fail(e1, "cudaEventCreateWithFlags"));
        b->side_done.push_back(ev);
    }
    if (b->cls.size() > 1) {
        cudaError_t e1 = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        if (e1 != cudaSuccess) return bail(cuda_fail(e1, "cudaEventCreateWithFlags"));
    }
    int rc;
    if ((rc = upload(&b->stab, stab, b->owned, s)) || (rc = upload(&b->titems, titems, b->owned, s)) ||
        (rc = upload(&b->litems, litems, b->owned, s)))
        return bail(rc);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamSynchronize"));
    *out = b;
    return PTYCHO_OK;
}

int ptycho_batch_size(const ptycho_batch_t *b, int32_t *n)
{
    if (!b || !n) return fail(PTYCHO_ERR_INVALID_ARG, "NULL argument");
    *n = (int32_t)b->plans.size();
    return PTYCHO_OK;
}

int ptycho_batch_member(const ptycho_batch_t *b, int32_t i, ptycho_plan_t **plan)
{
    if (!b || !plan || i < 0 || i >= (int32_t)b->plans.size())
        return fail(PTYCHO_ERR_INVALID_ARG, "bad batch member index");
    *plan = b->plans[i];
    return PTYCHO_OK;
}

int ptycho_batch_set_launch(ptycho_batch_t *b, int32_t variant, int32_t blocks_per_sm, ptycho_stream_t stream)
{
    if (!b) return fail(PTYCHO_ERR_INVALID_ARG, "batch is NULL");
    if (variant < 0 || variant >= PTYCHO_LAUNCH_VARIANTS) return fail(PTYCHO_ERR_INVALID_ARG, "variant out of range");
    if (blocks_per_sm < 0) return fail(PTYCHO_ERR_INVALID_ARG, "blocks_per_sm < 0");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<int> grids;
    for (const auto &c : b->cls) {
        int grid = 0;
        // the m = 64 class's 16 x 4 kernel keeps every block that fits (the
        // shape and cap are those of the two-stage kernels of the other classes);
        // m = 256 members take the variant through their own plans below
        if (c.m != 256)
            if (int rc = c.f4 ? f4_grid(2, c.n_items[0], &grid, 0)
                              : frame_update_grid(c.m, variant, c.n_items[variant], blocks_per_sm, &grid, nullptr))
                return rc;
        grids.push_back(grid);
    }
    // members iterate alone in the same shape, so their RF partials keep one layout
    for (auto *p : b->plans)
        if (int rc = apply_launch(p, variant, blocks_per_sm, s)) return rc;
    for (size_t i = 0; i < b->cls.size(); ++i) b->cls[i].grid = grids[i];
    b->variant = variant;
    b->blocks_per_sm = blocks_per_sm;
    drop_graphs(b->graph);
    return PTYCHO_OK;
}

int ptycho_batch_get_launch(const ptycho_batch_t *b, int32_t *variant, int32_t *blocks_per_sm)
{
    if (!b) return fail(PTYCHO_ERR_INVALID_ARG, "batch is NULL");
    if (variant) *variant = b->variant;
    if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
    return PTYCHO_OK;
}

// One iteration of every member: the frame updates of the probe-side classes
// are independent, so each class gets its own stream (parallel branches of the
// captured graph) and the subdomain update waits for all of them.
static int batch_enqueue(ptycho_batch_s *b, int parity, cudaStream_t s)
{
    const int nc = (int)b->cls.size();
    if (nc > 1) {
        OD2P_CUDA(cudaEventRecord(b->fork, s));
        for (int k = 1; k < nc; ++k) OD2P_CUDA(cudaStreamWaitEvent(b->side[k - 1], b->fork, 0));
    }
    for (int k = 0; k < nc; ++k) {
        const auto &c = b->cls[k];
        cudaStream_t sk = k == 0 ? s : b->side[k - 1];
        if (c.m == 256) {  // each member's waves (forking onto its own wave streams and joining back)
            for (auto *p : c.waves)
                if (int rc = launch_frame_update(p, sk)) return rc;
            continue;
        }
        if (int rc = c.f4 ? launch_frame_update_f4_table(c.tab, c.items[0], c.n_items[0], c.grid, parity, sk)
                          : launch_frame_update_table(c.m, b->variant, c.tab, c.items[b->variant],
                                                      c.n_items[b->variant], c.grid, parity, sk))
            return rc;
    }
    for (int k = 1; k < nc; ++k) {
        OD2P_CUDA(cudaEventRecord(b->side_done[k - 1], b->side[k - 1]));
        OD2P_CUDA(cudaStreamWaitEvent(s, b->side_done[k - 1], 0));
    }
    // blind members: the probe update of each (Algorithm 3 Steps 1, 3, 5), as in its own iteration
    for (auto *p : b->plans) {
        if (!p->blind) continue;
        if (int rc = launch_probe_avg(p, s)) return rc;
        if (int rc = launch_probe_reduce(p, nullptr, nullptr, s)) return rc;
        OD2P_CUDA(cudaMemcpyAsync(p->d_w, p->d_wnew, sizeof(float2) * p->MM, cudaMemcpyDeviceToDevice, s));
    }
    if (int rc = launch_subdomain_update_table(false, b->stab, b->titems, b->n_titems, parity, s)) return rc;
    return launch_subdomain_update_table(true, b->stab, b->litems, b->n_litems, parity, s);
}

int ptycho_batch_iterate(ptycho_batch_t *b, int32_t n_iter, ptycho_stream_t stream)
{
    if (!b) return fail(PTYCHO_ERR_INVALID_ARG, "batch is NULL");
    if (n_iter < 0) return fail(PTYCHO_ERR_INVALID_ARG, "n_iter < 0");
    for (auto *p : b->plans) {
        if (!p->initialised) return fail(PTYCHO_ERR_STATE, "od2p_init has not been called on every member");
        if (p->cur != b->cur) return fail(PTYCHO_ERR_STATE, "a member was iterated on its own");
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (int it = 0; it < n_iter; ++it) {
        const int par = b->cur;
        if (!b->graph[par]) {
            if (!b->cap_stream) OD2P_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
            OD2P_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
            int rc = batch_enqueue(b, par, b->cap_stream);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&b->graph[par], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                b->graph[par] = nullptr;
                return cuda_fail(e, "cudaGraphInstantiate");
            }
        }
        OD2P_CUDA(cudaGraphLaunch(b->graph[par], s));
        b->cur ^= 1;
        for (auto *p : b->plans) p->cur = b->cur;
    }
    return PTYCHO_OK;
}

}  // extern "C"

namespace od2p {

// A plan over the subdomains d with owner[d] == rank (see od2p.h); owner == null: all of them.
int build_plan(ptycho_plan_t **out, const ptycho_geometry *g, const float *f_dev, const int32_t *owner,
               int32_t rank, ptycho_stream_t stream)
{
    if (!out) return fail(PTYCHO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!g || !f_dev || !g->offsets_host) return fail(PTYCHO_ERR_INVALID_ARG, "NULL geometry, f or offsets");
    if (!supported_m(g->m)) return fail(PTYCHO_ERR_UNSUPPORTED, "probe side m must be 16, 32, 48, 64, 80, 96, 128 or 256");
    if (g->n_frames < 1 || g->img_h < g->m || g->img_w < g->m)
        return fail(PTYCHO_ERR_INVALID_ARG, "need n_frames >= 1 and an image at least m x m");
    if ((int64_t)g->img_h * g->img_w >= (1LL << 31))
        return fail(PTYCHO_ERR_UNSUPPORTED, "image larger than 2^31 pixels");
    if (g->sub_rows < 1 || g->sub_cols < 1 || g->sub_rows > g->img_h || g->sub_cols > g->img_w ||
        g->overlap_px < 0)
        return fail(PTYCHO_ERR_INVALID_ARG, "bad subdomain grid or overlap");
    if (!(g->eps > 0.f && g->eps < 1.f)) return fail(PTYCHO_ERR_INVALID_ARG, "eps must be in (0, 1)");
    if (!(g->eta > 0.f) || !(g->r >= 0.f) || !std::isfinite(g->eta) || !std::isfinite(g->r))
        return fail(PTYCHO_ERR_INVALID_ARG, "need eta > 0 and r >= 0");
    if (g->blind && (!(g->mu > 0.f) || !(g->gamma >= 0.f)))
        return fail(PTYCHO_ERR_INVALID_ARG, "blind plans need mu > 0 and gamma >= 0");
    const int m = g->m;
    if (int rc = check_geometry(g)) return rc;  // offsets (periodic: anywhere on the image)
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the decomposition always comes from every frame; a shard keeps the frames
    // of its own subdomains (ascending global index)
    std::vector<int32_t> all_offs(g->offsets_host, g->offsets_host + 2 * g->n_frames);
    const bool periodic = g->periodic != 0;
    Layout L = decompose(g->img_h, g->img_w, m, all_offs, g->sub_rows, g->sub_cols, g->overlap_px, periodic);
    if (int rc = check_periodic_rects(g, L)) return rc;
    const int D_all = g->sub_rows * g->sub_cols;
    std::vector<int32_t> sel;
    for (int j = 0; j < g->n_frames; ++j)
        if (!owner || owner[L.frame_sub[j]] == rank) sel.push_back(j);
    if (sel.empty()) return fail(PTYCHO_ERR_INVALID_ARG, "the shard's subdomains hold no frames");
    const int J = (int)sel.size();

    auto *p = new (std::nothrow) ptycho_plan_s();
    if (!p) return fail(PTYCHO_ERR_OOM, "host allocation failed");
    auto bail = [&](int rc) {
        ptycho_plan_destroy(p);
        return rc;
    };
    p->H = g->img_h;
    p->W = g->img_w;
    p->M = m;
    p->MM = m * m;
    p->J = J;
    p->sub_rows = g->sub_rows;
    p->sub_cols = g->sub_cols;
    p->overlap_px = g->overlap_px;
    p->eps = g->eps;
    p->eta = g->eta;
    p->r = g->r;
    p->mu = g->mu;
    p->gamma = g->gamma;
    p->blind = g->blind ? 1 : 0;
    p->periodic = periodic;
    p->img_rows = periodic ? p->H + m - 1 : p->H;
    p->img_cols = periodic ? p->W + m - 1 : p->W;
    p->offs.resize(2 * (size_t)J);
    p->frame_sub.resize(J);
    p->global_j = sel;
    for (int i = 0; i < J; ++i) {
        p->offs[2 * i] = L.placed[2 * sel[i]];
        p->offs[2 * i + 1] = L.placed[2 * sel[i] + 1];
        p->frame_sub[i] = L.frame_sub[sel[i]];
    }
    p->D = D_all;
    p->P = (int32_t)L.pair.size() / 2;
    if (owner) {
        p->owner.assign(owner, owner + D_all);
        p->rank = rank;
    }
    p->rect = L.rect;
    p->pair = L.pair;
    p->pair_rect = L.pair_rect;
    p->pair_shift = L.pair_shift;
    p->u_off.assign(p->D + 1, 0);
    for (int d = 0; d < p->D; ++d)
        p->u_off[d + 1] = p->u_off[d] + (int64_t)(p->rect[4 * d + 2] - p->rect[4 * d]) *
                                            (p->rect[4 * d + 3] - p->rect[4 * d + 1]);
    p->lam_off.assign(p->P + 1, 0);
    for (int k = 0; k < p->P; ++k)
        p->lam_off[k + 1] = p->lam_off[k] + (int64_t)(p->pair_rect[4 * k + 2] - p->pair_rect[4 * k]) *
                                                (p->pair_rect[4 * k + 3] - p->pair_rect[4 * k + 1]);
    p->u_len = p->u_off[p->D];
    p->lam_len = p->lam_off[p->P];
    // kernels index u, Lambda and the frame stacks with 32-bit integers
    if (p->u_len >= (1LL << 31) || p->lam_len >= (1LL << 31) || (int64_t)J * p->MM >= (1LL << 31))
        return bail(fail(PTYCHO_ERR_UNSUPPORTED, "subdomain, overlap or frame storage exceeds 2^31 elements"));

    // whole-image windows at the given offsets, in the image or its wrapped copy
    std::vector<int32_t> frame_base(J), frame_pitch(J), img_base(J), img_pitch(J, p->img_cols), img_offs(2 * (size_t)J);
    std::vector<std::vector<int32_t>> sub_frames(p->D), all_frames(1);
    for (int j = 0; j < J; ++j) {
        const int d = p->frame_sub[j];
        const int32_t *R = &p->rect[4 * d];
        frame_pitch[j] = R[3] - R[1];
        frame_base[j] = (int32_t)(p->u_off[d] + (int64_t)(p->offs[2 * j] - R[0]) * frame_pitch[j] +
                                  (p->offs[2 * j + 1] - R[1]));
        img_offs[2 * j] = all_offs[2 * sel[j]];
        img_offs[2 * j + 1] = all_offs[2 * sel[j] + 1];
        img_base[j] = img_offs[2 * j] * p->img_cols + img_offs[2 * j + 1];
        sub_frames[d].push_back(j);
        all_frames[0].push_back(j);
    }
    // neighbours of each subdomain: its pairs in list order (e ascending, then the
    // shift), each with its reverse pair and Omega_e moved into d's coordinates
    std::vector<int32_t> nbr_ptr(p->D + 1, 0), nbr;
    std::vector<int> rev, first;
    pair_links(L, rev, first);
    for (int k = 0; k < p->P; ++k) nbr.insert(nbr.end(), {p->pair[2 * k + 1], k, rev[k]});
    for (int k = 0, d = 0; d < p->D; ++d) {
        while (k < p->P && p->pair[2 * k] <= d) ++k;
        nbr_ptr[d + 1] = k;
    }
    std::vector<NbrInfo> nbr_info(nbr.size() / 3);
    for (int d = 0; d < p->D; ++d)
        for (int i = nbr_ptr[d]; i < nbr_ptr[d + 1]; ++i) {
            const int e = nbr[3 * i], kde = nbr[3 * i + 1], ked = nbr[3 * i + 2];
            const int sR = p->pair_shift[2 * kde] * p->H, sC = p->pair_shift[2 * kde + 1] * p->W;
            const int32_t *Re = &p->rect[4 * e], *Pr = &p->pair_rect[4 * kde];
            nbr_info[i] = NbrInfo{Re[0] + sR, Re[1] + sC, Re[2] + sR, Re[3] + sC, (int32_t)p->u_off[e], Re[3] - Re[1],
                                  Pr[0], Pr[1], Pr[3] - Pr[1], (int32_t)p->lam_off[kde],
                                  (int32_t)p->lam_off[ked], first[kde]};
        }
    // subdomain tiles: a shard tiles only its own subdomains (the others' rectangles
    // hold halo copies that the subdomain update reads but never writes)
    std::vector<int32_t> tile_rect = p->rect;
    if (owner)
        for (int d = 0; d < p->D; ++d)
            if (owner[d] != rank) tile_rect[4 * d + 2] = tile_rect[4 * d];
    HostTiles st = make_tiles(p->D, tile_rect, sub_frames, p->offs, m);
    // neighbours of each subdomain tile whose rectangle meets the tile
    std::vector<int32_t> tile_nbr_ptr(1, 0);
    std::vector<NbrInfo> tile_nbr;
    for (const Tile &t : st.tiles) {
        const int32_t *R = &p->rect[4 * t.reg];
        const int r0 = R[0] + t.r0, c0 = R[1] + t.c0;
        const int r1 = std::min(r0 + TILE_H, R[2]), c1 = std::min(c0 + TILE_W, R[3]);
        for (int i = nbr_ptr[t.reg]; i < nbr_ptr[t.reg + 1]; ++i) {
            const NbrInfo &nb = nbr_info[i];
            if (nb.r0 < r1 && r0 < nb.r1 && nb.c0 < c1 && c0 < nb.c1) tile_nbr.push_back(nb);
        }
        tile_nbr_ptr.push_back((int32_t)tile_nbr.size());
    }
    std::vector<TileInfo> tile_info;
    for (size_t t = 0; t < st.tiles.size(); ++t) {
        const Tile &T = st.tiles[t];
        const int32_t *R = &p->rect[4 * T.reg];
        const int wd = R[3] - R[1], hd = R[2] - R[0];
        tile_info.push_back(TileInfo{(int32_t)(p->u_off[T.reg] + (int64_t)T.r0 * wd + T.c0), wd,
                                     std::min(TILE_H, hd - T.r0), std::min(TILE_W, wd - T.c0), R[0] + T.r0,
                                     R[1] + T.c0, tile_nbr_ptr[t], tile_nbr_ptr[t + 1] - tile_nbr_ptr[t],
                                     st.ptr[t], st.ptr[t + 1] - st.ptr[t], T.reg, R[2]});
    }
    std::vector<int32_t> img_rect = {0, 0, p->img_rows, p->img_cols};
    HostTiles it = make_tiles(1, img_rect, all_frames, img_offs, m);
    if (periodic) {
        int rc0;
        if ((rc0 = dev_alloc(&p->d_upad, (size_t)p->img_rows * p->img_cols, p->owned, s)) ||
            (rc0 = dev_alloc(&p->d_gpad, (size_t)p->img_rows * p->img_cols, p->owned, s)))
            return bail(rc0);
    }

    auto &own = p->owned;
    const size_t JMM = (size_t)J * p->MM;
    int rc;
    if ((rc = upload(&p->d_offs, p->offs, own, s)) || (rc = upload(&p->d_frame_sub, p->frame_sub, own, s)) ||
        (rc = upload(&p->d_frame_base, frame_base, own, s)) ||
        (rc = upload(&p->d_frame_pitch, frame_pitch, own, s)) || (rc = upload(&p->d_img_base, img_base, own, s)) ||
        (rc = upload(&p->d_img_pitch, img_pitch, own, s)) ||
        (rc = upload(&p->d_rect, p->rect, own, s)) || (rc = upload(&p->d_nbr_ptr, nbr_ptr, own, s)) ||
        (rc = upload(&p->d_nbr, nbr, own, s)) || (rc = upload(&p->d_pair_rect, p->pair_rect, own, s)) ||
        (rc = upload(&p->d_pair, p->pair, own, s)) || (rc = upload(&p->d_pair_shift, p->pair_shift, own, s)) ||
        (rc = upload(&p->d_nbr_info, nbr_info, own, s)) ||
        (rc = upload(&p->d_u_off, p->u_off, own, s)) || (rc = upload(&p->d_lam_off, p->lam_off, own, s)) ||
        (rc = upload_tiles(p->sub_tiles, st, own, s)) || (rc = upload_tiles(p->img_tiles, it, own, s)) ||
        (rc = upload(&p->sub_tiles.nbr_ptr, tile_nbr_ptr, own, s)) ||
        (rc = upload(&p->sub_tiles.nbr, tile_nbr, own, s)) ||
        (rc = upload(&p->sub_tiles.info, tile_info, own, s)) ||
        (rc = upload_groups(p->sub_groups, sub_frames, own, s)) ||
        (rc = upload_groups(p->img_groups, all_frames, own, s)))
        return bail(rc);
    // twiddles exp(-2 pi i k / m), computed in double and rounded once
    std::vector<float2> tw(m);
    for (int k = 0; k < m; ++k) {
        const double a = -2.0 * 3.14159265358979323846 * (double)k / (double)m;
        tw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    if ((rc = upload(&p->d_tw, tw, own, s))) return bail(rc);
    if (p->blind && g->fourier_support_host) {
        std::vector<float> mask(p->MM);
        for (int k = 0; k < p->MM; ++k) mask[k] = g->fourier_support_host[k] ? 1.f : 0.f;
        p->has_mask = true;
        if ((rc = upload(&p->d_mask, mask, own, s))) return bail(rc);
    }
    p->n_rf_parts = rf_parts(m, J, 0);
    // RF partials sized for either launch shape of the frame update
    const int rf_cap = std::max(rf_parts(m, J, 0), rf_parts(m, J, 1));
    if ((rc = prepare_kernels(m)) ||
        (rc = frame_update_grid(m, 0, frame_groups(m, J, 0), 0, &p->n_k1_blocks, nullptr)))
        return bail(rc);
    p->n_loss_blocks = m == 256 ? J * 16 : (J + frames_per_block(m) - 1) / frames_per_block(m);
    const int n_chunks = std::max(p->sub_groups.n_chunks, p->img_groups.n_chunks);
    if ((rc = dev_alloc(&p->d_sqrtf, JMM, own, s)) || (rc = dev_alloc(&p->d_gamma, JMM, own, s)) ||
        (rc = dev_alloc(&p->d_q, JMM, own, s)) || (rc = dev_alloc(&p->d_u[0], p->u_len, own, s)) ||
        (rc = dev_alloc(&p->d_u[1], p->u_len, own, s)) || (rc = dev_alloc(&p->d_nrm, p->u_len, own, s)) ||
        (rc = dev_alloc(&p->d_lam[0], p->lam_len, own, s)) ||
        (rc = dev_alloc(&p->d_lam[1], p->lam_len, own, s)) || (rc = dev_alloc(&p->d_w, p->MM, own, s)) ||
        (rc = dev_alloc(&p->d_wnew, p->MM, own, s)) ||
        (rc = dev_alloc(&p->d_probe_part, (size_t)n_chunks * p->MM, own, s)) ||
        (rc = dev_alloc(&p->d_probe_part_n, (size_t)n_chunks * p->MM, own, s)) ||
        (rc = dev_alloc(&p->d_rf_part, rf_cap, own, s)) ||
        (rc = dev_alloc(&p->d_re_part, 2 * (size_t)p->sub_tiles.n_tiles, own, s)) ||
        (rc = dev_alloc(&p->d_loss_part, std::max(J, p->n_loss_blocks), own, s)) ||
        (rc = dev_alloc(&p->d_metrics, 5, own, s)) || (rc = dev_alloc(&p->d_err, 1, own, s)) ||
        (rc = dev_alloc(&p->d_rc_part, (size_t)(p->P + 1) * 64, own, s)) ||
        (rc = dev_alloc(&p->d_snr_part, 2 * 152 * 4, own, s)) || (rc = dev_alloc(&p->d_snr, 3, own, s)) ||
        (rc = dev_alloc(&p->d_opn, 2, own, s)) || (rc = dev_alloc(&p->d_until, 4, own, s)))
        return bail(rc);
    if (p->blind) {
        if ((rc = dev_alloc(&p->d_Wd, (size_t)p->D * p->MM, own, s)) || (rc = dev_alloc(&p->d_Delta, (size_t)p->D * p->MM, own, s)))
            return bail(rc);
    }
    if (m == 256)  // the default wave shape: chains of waves side by side, at most one per wave
        if ((rc = configure_waves(p, WAVE_256, WAVE_CHAINS_256, s))) return bail(rc);
    if (!p->blind) {
        // gather slots: ranks and counts on the device (one pass over the tile
        // lists), then the slot array sized by the largest count
        int32_t *d_setup = nullptr, h_setup[2] = {0, 0};
        if ((rc = dev_alloc(&p->d_rank, JMM, own, s)) || (rc = dev_alloc(&p->d_cnt, (size_t)p->u_len, own, s)) ||
            (rc = dev_alloc(&d_setup, 2, own, s)))
            return bail(rc);
        cudaError_t e1;
        if ((e1 = cudaMemsetAsync(p->d_cnt, 0, (size_t)p->u_len, s)) != cudaSuccess ||
            (e1 = cudaMemsetAsync(d_setup, 0, 2 * sizeof(int32_t), s)) != cudaSuccess)
            return bail(cuda_fail(e1, "cudaMemsetAsync"));
        if ((rc = launch_slot_rank(p, d_setup, s))) return bail(rc);
        if ((e1 = cudaMemcpyAsync(h_setup, d_setup, sizeof(h_setup), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e1 = cudaStreamSynchronize(s)) != cudaSuccess)
            return bail(cuda_fail(e1, "slot ranks"));
        p->slot_k = h_setup[1];
        p->slots = !h_setup[0] && (int64_t)p->slot_k * p->u_len < (1LL << 32);
        if (p->slots && (rc = dev_alloc(&p->d_slot, (size_t)std::max(p->slot_k, 1) * p->u_len, own, s)))
            return bail(rc);
    }
    cudaError_t e;
    if ((e = cudaMemsetAsync(p->d_metrics, 0, 5 * sizeof(double), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->d_rf_part, 0, sizeof(float) * rf_cap, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->d_re_part, 0, sizeof(float) * 2 * p->sub_tiles.n_tiles, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->d_w, 0, sizeof(float2) * p->MM, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->d_err, 0, sizeof(int32_t), s)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMemsetAsync"));
    // kernel argument tables (buffer pointers are fixed from here on)
    fill_frame_args(p, p->h_fargs);
    fill_sub_args(p, p->h_sargs);
    {
        std::vector<FrameArgs> fa(p->h_fargs, p->h_fargs + 2);
        std::vector<SubArgs> sa(p->h_sargs, p->h_sargs + 2);
        if ((rc = upload(&p->d_fargs, fa, own, s)) || (rc = upload(&p->d_sargs, sa, own, s))) return bail(rc);
    }
    if ((rc = launch_ingest_f(p, f_dev, s)) || (rc = launch_sum_sqrtf(p, s))) return bail(rc);
    // Step 0 with u = 1 and a zero probe until od2p_init
    if ((rc = launch_init_state(p, nullptr, p->d_w, s))) return bail(rc);
    if ((e = cudaMemsetAsync(p->d_gamma, 0, sizeof(float2) * JMM, s)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMemsetAsync"));
    if (owner && (rc = build_halo_tables(p, s))) return bail(rc);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bail(cuda_fail(e, "cudaStreamSynchronize"));
    *out = p;
    return PTYCHO_OK;
}

}  // namespace od2p

