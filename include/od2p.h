/*
 * od2p.h -- C ABI of the GB300 (sm_103a) OD2P ptychography library.
 *
 * Method: Chang, Glowinski, Marchesini, Tai, Wang, Zeng, "Overlapping Domain
 * Decomposition Methods for Ptychographic Imaging", arXiv:2011.00162.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Complex data are interleaved single precision (ptycho_c32 = {re, im}),
 *    row-major.  Frames are J x m x m, contiguous.  Images are img_h x img_w.
 *  - The 2-D DFT F is unitary (1/m both ways) with frequencies in natural
 *    (unshifted) order (section 2: "normalized discrete Fourier transform").
 *  - Scan offsets are the (row, col) of the top-left pixel of each m x m
 *    window; S_j cuts that window without wrap-around (section 4 set-up).
 *  - Pointers named *_dev are device pointers owned by the caller; pointers
 *    named *_host are host pointers owned by the caller.  Nothing crosses the
 *    ABI by ownership transfer except the opaque plan, which the caller frees
 *    with ptycho_plan_destroy.
 *  - Every call enqueues its GPU work on `stream` (a cudaStream_t; NULL is the
 *    legacy default stream) and returns without synchronising unless it says
 *    otherwise.  Plan-owned state may only be used from one stream at a time.
 *  - Every call returns PTYCHO_OK (0) or an error code; ptycho_last_error()
 *    returns a message for the calling thread.  No C++ exception crosses the
 *    ABI and no call aborts the process.
 *  - Supported probe sides m: 16, 32, 64, 128, 256 and the mixed-radix sides
 *    48 (8 x 6), 80 (16 x 5) and 96 (8 x 12) -- the paper fixes no size, and
 *    detectors are not limited to powers of two.  Up to 128 a frame is
 *    transformed in one thread block's shared memory; 256 x 256 frames go
 *    through row / column / row passes over a plan-owned intermediate, in
 *    waves small enough to stay in L2 (the frame update can instead hold each
 *    frame in the distributed shared memory of a cluster of 16 thread blocks,
 *    launch variant 1).  Other m return PTYCHO_ERR_UNSUPPORTED
 *    (stagm_loss_noalloc: 16, 32, 64, 128).
 */
#ifndef OD2P_H
#define OD2P_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t without including the CUDA headers. */
typedef struct CUstream_st *ptycho_stream_t;

typedef struct {
    float re, im;
} ptycho_c32;

enum {
    PTYCHO_OK = 0,
    PTYCHO_ERR_INVALID_ARG = 1, /* a size, pointer, offset or parameter is out of range   */
    PTYCHO_ERR_UNSUPPORTED = 2, /* valid but not implemented (e.g. m not in {16..256})    */
    PTYCHO_ERR_OOM = 3,         /* device or host allocation failed                       */
    PTYCHO_ERR_CUDA = 4,        /* a CUDA runtime call failed (message has the CUDA text) */
    PTYCHO_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up                     */
    PTYCHO_ERR_STATE = 6        /* call not valid in the plan's current state             */
};

/* od2p_get_state / od2p_set_state selectors */
enum {
    PTYCHO_STATE_U = 0,      /* u_d: concatenated subdomain rectangles, d ascending        */
    PTYCHO_STATE_GAMMA = 1,  /* Gamma: J x m x m, natural frequency order                  */
    PTYCHO_STATE_LAMBDA = 2, /* Lambda_{d,e}: concatenated pair rectangles, pair order     */
    PTYCHO_STATE_WD = 3,     /* W_d: D x m x m per-subdomain probe copies (blind)          */
    PTYCHO_STATE_DELTA = 4,  /* Delta_d: D x m x m multipliers of W_d = w (blind)          */
    PTYCHO_STATE_W = 5,      /* w: m x m shared probe                                      */
    PTYCHO_STATE_Q = 6       /* last frame residual q_j = F^*(z_j - Gamma_j), times conj(w) in nonblind
                                plans (J x m x m, spatial), read-only */
};

/* overlap_add flags */
enum {
    PTYCHO_OA_IFFT = 1 /* apply F^* to each frame first, so the call computes A^* y */
};

/*
 * Problem description (section 2, problem PtychoPR; sections 2.1 and 3.1 for
 * the decomposition; section 2.2 for eps; Algorithms 1-3 for eta, r, mu, gamma).
 *
 * Decomposition rule (the paper builds subdomains from complete frames but does
 * not fix a rule for 2-D grids): the image is cut into sub_rows x sub_cols
 * core tiles at floor(k*H/sub_rows), floor(k*W/sub_cols); frame j joins the
 * tile containing its window centre offs[j] + (m-1)/2; Omega_d is the bounding
 * box of its core tile grown by ceil(overlap_px/2) on interior sides (clipped)
 * and of its frames' windows.  Ordered pairs (d, e) with intersecting Omega
 * carry Lambda_{d,e}; sorted by (d, e).
 *
 * Periodic boundaries (periodic = 1; section 4 names them as the usual
 * alternative to its vacuum boundary of ones, and does not decompose a
 * periodic image -- this is a reading): the image is a torus and window j
 * covers pixels ((offs[j] + a) mod img_h, (offs[j] + b) mod img_w), offsets
 * anywhere in [0, img_h) x [0, img_w).  Rectangles then live in extended
 * coordinates (pixel (R, C) is image pixel (R mod img_h, C mod img_w)): every
 * core tile grows on all sides and is not clipped, frame j is placed at the
 * copy of its offset whose doubled centre 2 o + m - 1 lies in [0, 2 img_h) x
 * [0, 2 img_w) (offs - img_h where it would not) and joins that centre's tile,
 * and the pairs are (d, e, s) for shifts s in {-2, ..., 2}^2 periods such that
 * Omega_d meets Omega_e moved by s (d = e included, s != 0), sorted by
 * (d, e, s_r, s_c), each kept in d's coordinates -- (e, d, -s) is the same
 * region seen from e.  A rectangle must stay within (-img_h, 2 img_h) x
 * (-img_w, 2 img_w) (INVALID_ARG otherwise).  Step 0 reads u0 modulo the
 * image and od2p_merge / od2p_snr average every copy of a pixel.  The
 * image-space operators (ptycho_forward, overlap_add, stagm_loss_grad) read
 * whole-image windows from a plan-owned wrapped copy of (img_h + m - 1) x
 * (img_w + m - 1) pixels and add their adjoints into the same grid, whose
 * copies of each pixel are then summed onto the image in a fixed order.
 * Shards exchange the same messages, pair by pair (a pair with both ends on
 * one rank, a subdomain's pair with itself included, sends nothing).
 */
typedef struct {
    int32_t img_h, img_w;           /* image size in pixels                                 */
    int32_t m;                      /* probe side: 16, 32, 48, 64, 80, 96, 128 or 256      */
    int32_t n_frames;               /* J >= 1                                              */
    const int32_t *offsets_host;    /* J x 2 (row, col), 0 <= row <= img_h-m, col likewise
                                       (periodic: 0 <= row < img_h, col likewise)          */
    int32_t sub_rows, sub_cols;     /* subdomain grid, >= 1                                */
    int32_t overlap_px;             /* requested minimum overlap width, >= 0               */
    float eps;                      /* ST-AGM truncation, 0 < eps < 1 (paper: 0.5)         */
    float eta;                      /* ADMM penalty on A_d u_d = z_d, > 0                  */
    float r;                        /* ADMM penalty on overlap continuity, >= 0            */
    float mu;                       /* blind: penalty on W_d = w, > 0 when blind           */
    float gamma;                    /* blind: proximal weight of the U-update, >= 0        */
    int32_t blind;                  /* 0: Algorithm 2 (known probe); 1: Algorithm 3        */
    const uint8_t *fourier_support_host; /* blind: m x m, 1 on the support of F w; NULL = all */
    int32_t periodic;               /* 0: vacuum boundary (section 4); 1: periodic (above) */
} ptycho_geometry;

typedef struct ptycho_plan_s ptycho_plan_t;

/* Message of the last failing call on this thread ("" if none). Never NULL. */
const char *ptycho_last_error(void);

/* ABI version, incremented on incompatible changes. */
int32_t ptycho_abi_version(void);

/*
 * Device memory of plans and batches comes from one stream-ordered pool per
 * device that keeps memory freed by ptycho_plan_destroy / ptycho_batch_destroy
 * for the next plan, so repeated reconstructions of one workload allocate
 * nothing new from the driver.  This call synchronises the current device and
 * returns the pool's unused memory to the driver (memory of live plans stays).
 * Errors: CUDA, UNSUPPORTED (device ordinal above 63).
 */
int ptycho_release_cached_memory(void);

/*
 * Build a plan: validate g, compute the decomposition, allocate plan-owned
 * device state, and ingest the measured intensities f (J x m x m FP32,
 * natural frequency order, f >= 0).  f_dev is read during this call only (the
 * plan keeps sqrt(f) in its own layout).  The state is initialised as Step 0
 * of Algorithms 1-3 with u = 1 and the probe all zeros; call od2p_init before
 * iterating.  On error *out is set to NULL and nothing is leaked.
 * Nonblind plans add the A_d^* summands of eq. (Alg1-solver-u) through
 * per-pixel gather slots (each frame writes its conj(w)-weighted residual to
 * the slot of its rank among the frames covering the pixel; the subdomain
 * update sums a pixel's slots in ascending j).  When more than 255 frames
 * cover one pixel, or the slots would exceed 2^32 elements, the plan uses the
 * frame-list gather of blind plans instead, weighting with the known probe:
 * the same result up to rounding, at a lower speed.
 * Errors: INVALID_ARG (NULL pointer, bad sizes/offsets/parameters),
 * UNSUPPORTED (m), OOM, CUDA.
 */
int ptycho_plan(ptycho_plan_t **out, const ptycho_geometry *g, const float *f_dev,
                ptycho_stream_t stream);

/*
 * The decomposition alone, on the host (no device work): frame_sub_host[J]
 * receives each frame's subdomain and rect_host[D*4] (D = sub_rows *
 * sub_cols) each subdomain's rectangle (r0, c0, r1, c1), half-open, by the
 * rule stated above.  Either output may be NULL.  Used to split a problem
 * over ranks before any plan exists.  Errors: INVALID_ARG, UNSUPPORTED (m).
 */
int ptycho_decompose(const ptycho_geometry *g, int32_t *frame_sub_host, int32_t *rect_host);

/*
 * Subdomain sharding of one reconstruction over several ranks (section 3.1:
 * the subdomain problems are coupled only through their overlaps).  A shard
 * plan holds the subdomains d with owner_host[d] == rank (owner_host: D ranks,
 * host memory) -- their frames, u_d, Lambda_{d,e} and, blind, W_d and Delta_d
 * -- and halo copies of every other subdomain's u, Lambda, W and Delta in the
 * same layouts as a whole plan (od2p_state_len, od2p_get_state).  f_dev holds
 * the intensities of the shard's own frames only (those j with
 * owner[frame_sub[j]] == rank, ascending j; ptycho_decompose gives
 * frame_sub), J_shard x m x m.  od2p_init, od2p_iterate and the stage calls
 * then update only the shard's own values, each computed exactly as in the
 * whole plan, provided the halo copies are current before every iteration:
 * between iterations each rank packs, for every peer, the strips of its own
 * u_e on the overlaps with the peer's subdomains and its Lambda_{e,d} (blind:
 * also its W_e and Delta_e), moves the message to the peer (NCCL, MPI or
 * host memory: the library does not communicate), and unpacks what it
 * receives.  Message order (both sides derive it from the decomposition): for
 * every ordered pair (e, d) in pair order with owner[e] = sender and owner[d]
 * = receiver, the rows of u_e on Omega_e n Omega_d, then Lambda_{e,d}
 * (row-major); blind, then W_e and Delta_e (m x m) of every e the sender owns,
 * e ascending.  A shard's od2p_metrics covers its own frames and subdomains;
 * its merge and its halo state are only as current as the last unpack.
 * Errors: INVALID_ARG (owner out of [0, D), a rank owning no subdomain or no
 * frame), and as ptycho_plan.
 */
int ptycho_plan_shard(ptycho_plan_t **out, const ptycho_geometry *g, const int32_t *owner_host, int32_t rank,
                      const float *f_dev, ptycho_stream_t stream);
/* Number of frames a plan holds and, for a shard, their global indices
 * (global_index_host: n_frames entries; a whole plan gives 0 .. J-1).     */
int ptycho_plan_frames(const ptycho_plan_t *plan, int32_t *n_frames, int32_t *global_index_host);
/* Complex elements of the halo messages to and from `peer` (any output may be
 * NULL).  Errors: INVALID_ARG (peer out of range or the shard's own rank),
 * STATE (not a shard).                                                     */
int od2p_halo_size(const ptycho_plan_t *plan, int32_t peer, int64_t *send_elems, int64_t *recv_elems);
/* Write the message for `peer` from the shard's current state into send_dev
 * (device, od2p_halo_size's send_elems complex), or write the message
 * received from `peer` (recv_dev, recv_elems) into the shard's halo copies.
 * Asynchronous on `stream`; call them between iterations.  Errors: as
 * od2p_halo_size, INVALID_ARG (NULL buffer for a non-empty message), CUDA.  */
int od2p_halo_pack(const ptycho_plan_t *plan, int32_t peer, ptycho_c32 *send_dev, ptycho_stream_t stream);
int od2p_halo_unpack(ptycho_plan_t *plan, int32_t peer, const ptycho_c32 *recv_dev, ptycho_stream_t stream);

/* Free a plan and everything it owns (synchronises the device). NULL is a no-op. */
int ptycho_plan_destroy(ptycho_plan_t *plan);

/* Sizes of the decomposition: subdomains D, ordered pairs P, and the element
 * counts of the concatenated u and Lambda layouts.  Any output may be NULL.  */
int ptycho_plan_dims(const ptycho_plan_t *plan, int32_t *n_sub, int32_t *n_pairs,
                     int64_t *u_len, int64_t *lambda_len);

/* Host copies of the decomposition: frame_sub[J], rect[D*4] = (r0, c0, r1, c1)
 * half-open, pair[P*2] = (d, e), pair_rect[P*4].  Any output may be NULL.     */
int ptycho_plan_layout(const ptycho_plan_t *plan, int32_t *frame_sub_host, int32_t *rect_host,
                       int32_t *pair_host, int32_t *pair_rect_host);
/* Each pair's shift pair_shift[P*2] = (s_r, s_c) in periods (all 0 without
 * periodic boundaries) and each frame's placed offset placed[J*2] in extended
 * coordinates (the given offset without periodic boundaries).  Any output may
 * be NULL.  Errors: INVALID_ARG (plan NULL).                                  */
int ptycho_plan_periodic_layout(const ptycho_plan_t *plan, int32_t *pair_shift_host, int32_t *placed_host);

/*
 * Forward operator (section 2, operator A): frames_out[j] = F(w o S_j u) for
 * every frame of the plan.  u_dev: img_h x img_w; w_dev: m x m;
 * frames_out_dev: J x m x m (natural frequency order).  Errors: INVALID_ARG.
 */
int ptycho_forward(const ptycho_plan_t *plan, const ptycho_c32 *u_dev, const ptycho_c32 *w_dev,
                   ptycho_c32 *frames_out_dev, ptycho_stream_t stream);

/*
 * Proximal map of the ST-AGM (section 2.2, eq. Prox_sol), elementwise:
 * z[i] = argmin_z g_eps(z; f[i]) + lambda/2 |z - y[i]|^2.  The threshold is
 * read as |y| < (eps - (1-eps)/lambda) sqrt(f) (the paper's is garbled);
 * sign(0) = 1.  y, z: n complex; f: n floats >= 0; z may alias y.
 * Errors: INVALID_ARG (n < 0, NULL with n > 0, eps not in (0,1), lambda <= 0).
 */
int stagm_prox(const ptycho_c32 *y_dev, const float *f_dev, ptycho_c32 *z_dev, int64_t n,
               float eps, float lambda, ptycho_stream_t stream);

/*
 * Overlap-add (the adjoint A^* of section 2, used by eq. Alg1-solver-u):
 * image_out = sum_j S_j^T (conj(w) o G_j), G_j = F^* frames_j when flags has
 * PTYCHO_OA_IFFT, else frames_j.  Each pixel sums the frames covering it in
 * ascending j with no atomics, so the result is bitwise reproducible.
 * frames_dev: J x m x m; w_dev: m x m; image_out_dev: img_h x img_w
 * (overwritten; uncovered pixels are 0).  Uses the plan's frame scratch, so
 * calls on one plan must not overlap.  Errors: INVALID_ARG.
 */
int overlap_add(ptycho_plan_t *plan, const ptycho_c32 *frames_dev, const ptycho_c32 *w_dev,
                ptycho_c32 *image_out_dev, int32_t flags, ptycho_stream_t stream);

/*
 * Step 0 of Algorithms 1-3: u_d = R_d u0 (u0_dev img_h x img_w, or NULL for
 * all ones), Gamma = Lambda = 0; the probe w (and, blind, every W_d) = w0_dev
 * (m x m, required), Delta = 0.  Errors: INVALID_ARG.
 */
int od2p_init(ptycho_plan_t *plan, const ptycho_c32 *u0_dev, const ptycho_c32 *w0_dev,
              ptycho_stream_t stream);

/*
 * One ADMM iteration: Algorithm 2 Steps 1-4 (nonblind; D = 2 is Algorithm 1)
 * or Algorithm 3 Steps 1-5 (blind), repeated n_iter times.  The iteration is
 * replayed from a CUDA graph captured on first use.  Errors: INVALID_ARG
 * (n_iter < 0), STATE (od2p_init not called), CUDA.
 */
int od2p_iterate(ptycho_plan_t *plan, int32_t n_iter, ptycho_stream_t stream);

/*
 * Iterate until section 4's stopping test holds: after every iteration the RF
 * of that iteration (the same fixed-order sum as od2p_metrics) is compared on
 * the device, and the loop stops after the first iteration with
 * (float) RF <= rf_tol, or after max_iter iterations.  The loop runs inside
 * one CUDA graph (a conditional while node over two iterations, the second
 * behind a conditional if), so no iteration waits for the host; at least one
 * iteration runs when max_iter > 0.  Writes the iterations done and the last
 * RF to the host (either may be NULL) and synchronises `stream`.  The result
 * equals od2p_iterate one iteration at a time with od2p_metrics after each.
 * Errors: INVALID_ARG (max_iter < 0, tol not finite), STATE (before
 * od2p_init, or a batch member), CUDA.
 */
int od2p_iterate_until(ptycho_plan_t *plan, float rf_tol, int32_t max_iter, int32_t *n_done_host,
                       float *rf_host, ptycho_stream_t stream);

/*
 * The two halves of one nonblind iteration, for stage timing:
 *  od2p_frame_update:     Steps 1-2 frame part -- z = Prox(Gamma + A_d u_d),
 *                         Gamma += A_d u_d - z, q_j = conj(w) o F^*(z - Gamma)
 *                         (eqs. updateZ, updateM-1-multi); fused per frame.
 *  od2p_subdomain_update: Step 1 v (eq. updateV-multi), Step 3 u (eq.
 *                         Alg1-solver-u, D-subdomain form) by gathering q_j in
 *                         ascending j, Step 4 Lambda (eq. updateM-2-multi).
 * Calling them in this order equals od2p_iterate(plan, 1) for a nonblind
 * plan; for a blind plan, frame update, probe_update and subdomain update in
 * that order do (the frame update then stores the unweighted residual and the
 * subdomain update weights it with W_d).  Errors: STATE (od2p_init not
 * called), CUDA.
 */
int od2p_frame_update(ptycho_plan_t *plan, ptycho_stream_t stream);
int od2p_subdomain_update(ptycho_plan_t *plan, ptycho_stream_t stream);

/*
 * Blind probe update (Algorithm 3 Steps 1 (w), 3 (W) and 5 (Delta); eqs.
 * blind_w, blind_W, admm_Delta) from the frame residuals of the last frame
 * update.  od2p_iterate calls it for blind plans; exposed for stage timing.
 * Errors: STATE (nonblind plan, or od2p_init not called).
 */
int probe_update(ptycho_plan_t *plan, ptycho_stream_t stream);

/*
 * Merge of the subdomain solutions (section 4 set-up): pixels in one subdomain
 * keep their value, overlaps are averaged.  u_out_dev: img_h x img_w.
 */
int od2p_merge(const ptycho_plan_t *plan, ptycho_c32 *u_out_dev, ptycho_stream_t stream);

/*
 * Stopping metrics of section 4 from the last iteration, reduced in a fixed
 * order: RF of the iterate that entered it (sum |(|A_d u_d| - sqrt f)| /
 * sum sqrt f; blind: with W_d^n in place of w) and RE = max_d ||u_d^{n+1} -
 * u_d^n|| / ||u_d^{n+1}||.  loss: the ST-AGM data term of the current iterate
 * (eq. STAGM summed over frames, G_eps(B_d(W_d, u_d)); f_j), each frame taken
 * from its own subdomain copy u_d and probe (w, or W_d when blind): one extra
 * pass over the frames, made only when loss_host is not NULL; it uses the
 * loss scratch of stagm_loss_grad and leaves every state array unchanged.
 * Writes host scalars and synchronises `stream`.  Any output may be NULL.
 * Errors: INVALID_ARG, STATE (loss before od2p_init), TIMEOUT (a bounded wait
 * of an earlier frame update gave up), CUDA.
 */
int od2p_metrics(ptycho_plan_t *plan, float *rf_host, float *re_host, float *loss_host, ptycho_stream_t stream);

/*
 * Penalty changes between iterations (the paper fixes eta and r for a run and
 * names their automatic choice future work, section 4.3).  Gamma and Lambda are
 * the scaled multipliers of the augmented Lagrangian, so a change keeps the
 * unscaled ones: Gamma <- (eta_old / eta) Gamma, Lambda <- (r_old / r) Lambda
 * (the rescaling of Boyd, Parikh, Chu, Peleato, Eckstein 2011, 3.4.1; Lambda
 * is left alone when r = 0).  Drops the captured iteration graphs and
 * synchronises `stream`.  Errors: INVALID_ARG (eta <= 0, r < 0, not finite),
 * STATE (a batch member), CUDA.
 */
int od2p_set_penalties(ptycho_plan_t *plan, float eta, float r, ptycho_stream_t stream);

/*
 * Consensus residual of the current iterate: ||u_d - u_e|| summed over every
 * ordered pair's overlap, relative to ||u|| over all subdomain pixels (0 with
 * no pairs), reduced in a fixed order -- the primal residual of the consensus
 * constraint v = pi u_d = pi u_e of eq. (updateV-multi).  Writes a host float
 * and synchronises `stream`.  Errors: INVALID_ARG, CUDA.
 */
int od2p_consensus_residual(ptycho_plan_t *plan, float *rc_host, ptycho_stream_t stream);

/*
 * Primal residual of the frame constraint z_j = A_j u (Algorithm 2 Step 2: the
 * scaled multiplier moves by A_d u_d^n - z^{n+1}): od2p_gamma_snapshot copies
 * Gamma into plan-owned memory (allocated on first use), and
 * od2p_frame_residual returns ||Gamma - Gamma_snapshot|| / ||sqrt f|| over all
 * frame pixels, reduced in a fixed order.  Taken around one iteration, this is
 * the relative primal residual of that iteration.  od2p_frame_residual writes a
 * host float and synchronises `stream`.  Errors: INVALID_ARG, STATE (no
 * snapshot yet), OOM, CUDA.
 */
int od2p_gamma_snapshot(ptycho_plan_t *plan, ptycho_stream_t stream);
int od2p_frame_residual(ptycho_plan_t *plan, float *res_host, ptycho_stream_t stream);

/*
 * Measurement probes for the ceilings the frame update is compared with (the
 * paper has none): kind PTYCHO_PROBE_FMA runs n_blocks x 256 threads of eight
 * independent FP32 FMA chains for `iters` steps (16 FLOP per thread and step);
 * PTYCHO_PROBE_SMEM has each thread read eight conflict-free 16-byte shared-
 * memory words per step (128 bytes per thread and step).  One float per thread
 * goes to sink_dev (n_blocks x 256 floats, caller-owned).  Asynchronous on
 * `stream`; time it with events.  Errors: INVALID_ARG, CUDA.
 */
#define PTYCHO_PROBE_FMA 0
#define PTYCHO_PROBE_SMEM 1
int ptycho_peak_probe(int32_t kind, int32_t n_blocks, int32_t iters, float *sink_dev, ptycho_stream_t stream);

/*
 * The operator norms of Lemma 2.4's parameter set K (eq. paramsSet), taken over
 * all subdomains and ordered overlap pairs: norms_host[0] = max_d ||A_d^* A_d||
 * and norms_host[1] = max_{(d,e)} ||pi_{d,e} A_d^*||^2 (0 without overlaps).
 * A_d^* A_d is diagonal (eq. AtA), so these are the largest illumination
 * sum_j S_j^T |w|^2 over Omega_d and over Omega_d n Omega_e.  Nonblind plans
 * only (the known probe of od2p_init); synchronises `stream`.
 * Errors: INVALID_ARG, STATE (blind plan, or before od2p_init), CUDA.
 */
int od2p_operator_norms(ptycho_plan_t *plan, float *norms_host, ptycho_stream_t stream);

/*
 * Section 4's signal-to-noise ratio of the current recovery against the ground
 * truth: SNR(u_r, u_g) = -10 log10(||e^{i theta} u_r - u_g||^2 / ||u_r||^2) dB,
 * with u_r the merged image (as od2p_merge), u_g = truth_dev (img_h x img_w) and
 * theta = arg sum conj(u_r) u_g removing the recovery's global phase.
 * mask_dev: NULL (every pixel) or img_h x img_w bytes, nonzero where the pixel
 * counts (e.g. the illuminated pixels).  Two fixed-order reduction passes;
 * writes a host float and synchronises `stream`; the value is NaN when no
 * pixel is selected or the recovery is zero there.  Errors: INVALID_ARG, CUDA.
 */
int od2p_snr(ptycho_plan_t *plan, const ptycho_c32 *truth_dev, const uint8_t *mask_dev, float *snr_host,
             ptycho_stream_t stream);

/*
 * Data-driven initial probe of the blind experiments (section 4.2):
 * w0 = (1/J) sum_j F^* sqrt(f_j), from the intensities the plan holds.  The GPU
 * forms F^* of the mean amplitude (equal by linearity): the amplitudes are
 * averaged per frequency in ascending j with compensated FP32 addition, then
 * inverse-transformed by direct (unitary) DFT sums.  w0_dev: m x m, written.
 * Uses plan scratch (the frame-residual and probe buffers): do not overlap with
 * other calls on the plan.  Pass the result to od2p_init as w0 for a blind run.
 * Errors: INVALID_ARG, CUDA.
 */
int ptycho_probe_init(ptycho_plan_t *plan, ptycho_c32 *w0_dev, ptycho_stream_t stream);

/*
 * Launch shape of the frame update (the paper fixes none).  For m <= 128 two
 * shapes are compiled, each a (frames per block, threads per block) pair:
 *   m = 16: variant 0 (8, 256), variant 1 (4, 128);  m = 32: (4, 256), (2, 128);
 *   m = 64: (1, 512), (1, 512);  m = 128: (1, 1024), (1, 512);
 *   m = 48: (2, 384), (1, 384);  m = 80: (1, 448), (1, 640);  m = 96: (1, 384), (1, 768).
 * At m = 32, 48 and 64 variant 1 reads Gamma from L2 instead of staging it in
 * shared memory and is compiled for more resident blocks per SM.
 * The persistent kernel runs min(frame groups, b x SMs) blocks, b =
 * blocks_per_sm capped at what fits (0: as many as fit).  Every shape gives
 * the same iterates bit for bit; only the RF partial sums are grouped
 * differently.  m = 256 (blocks_per_sm ignored): variant 0 runs the row /
 * column / row passes over the plan's L2-resident intermediate; variant 1
 * transforms each frame in one pass inside a cluster of 16 thread blocks that
 * holds the frame in their distributed shared memory.  The two are the same
 * arithmetic in a different kernel sequence: iterates equal up to FP32
 * rounding (each is compared with the FP64 oracle), RF grouped alike.
 * ptycho_plan_set_launch drops the plan's captured iteration graphs (they are
 * recaptured on the next od2p_iterate); when the shape changes, RF reads 0
 * until the next frame update.  A batch member returns PTYCHO_ERR_STATE: use
 * ptycho_batch_set_launch.  ptycho_plan_get_launch reports the current shape
 * and the most blocks of it that fit on one SM (any output may be NULL).
 * Errors: INVALID_ARG (variant outside [0, PTYCHO_LAUNCH_VARIANTS) or
 * blocks_per_sm < 0), STATE, CUDA.
 */
#define PTYCHO_LAUNCH_VARIANTS 2

/*
 * Factorisation of the frame update's 64-point transforms (m = 64 only; the
 * paper fixes none): kind 0 (default) splits each axis 8 x 8 -- three shared-
 * memory exchanges per direction, the launch shapes above; kinds 1 and 2 split
 * each axis 16 x 4 and run both axes' radix-4 stages together in a 4 x 4 block
 * per thread -- two exchanges per direction, one frame per 256-thread block,
 * Gamma staged in shared memory (1) or read through L2 (2).  Kinds give the
 * same iterates up to FP32 rounding (not bit for bit); a plan's own iterates
 * stay deterministic.  Drops the captured graphs.  Errors: INVALID_ARG (kind
 * not 0-2), UNSUPPORTED (kind 1 or 2 with m != 64), STATE (a batch member).
 */
int ptycho_plan_set_fft(ptycho_plan_t *plan, int32_t kind, ptycho_stream_t stream);
int ptycho_plan_get_fft(const ptycho_plan_t *plan, int32_t *kind);
int ptycho_plan_set_launch(ptycho_plan_t *plan, int32_t variant, int32_t blocks_per_sm, ptycho_stream_t stream);
int ptycho_plan_get_launch(const ptycho_plan_t *plan, int32_t *variant, int32_t *blocks_per_sm,
                           int32_t *max_blocks_per_sm);
/*
 * How the frame update is launched (the paper has no counterpart; Step 1 of
 * Algorithms 2 and 3 runs over all frames at once).  m = 256 with launch
 * variant 0 moves the frames through its three passes in waves of
 * *wave_frames frames, the waves dealt round-robin to *chains chains that run
 * side by side on streams of the plan (forked from and joined back into the
 * caller's stream), 3 launches per wave; every other shape reports 0, 1 and one
 * launch.  *launches: kernel launches of one frame update.  Any output may be
 * NULL.  Errors: INVALID_ARG (plan NULL).
 */
int ptycho_plan_get_waves(const ptycho_plan_t *plan, int32_t *wave_frames, int32_t *chains, int32_t *launches);
/* m = 256: frames per wave (1 .. 152) and chains of waves side by side (1 .. 8;
 * at most one per wave) for launch variant 0 (default 19 frames, 4 chains).
 * Every shape gives the same iterates bit for bit; the plan grows its
 * intermediate (chains x wave_frames frames of 512 KB) and makes streams as
 * needed.  Drops the captured graphs.  Errors: INVALID_ARG, UNSUPPORTED
 * (m != 256), OOM.                                                            */
int ptycho_plan_set_waves(ptycho_plan_t *plan, int32_t wave_frames, int32_t chains, ptycho_stream_t stream);

/* Element count (complex) of a state selector (PTYCHO_STATE_*). */
int od2p_state_len(const ptycho_plan_t *plan, int32_t which, int64_t *n_out);

/* Copy state out of / into the plan (device buffers of od2p_state_len
 * elements, layouts as documented at PTYCHO_STATE_*).  Used for checkpoint /
 * resume and parity checks.  PTYCHO_STATE_Q cannot be set.                   */
int od2p_get_state(const ptycho_plan_t *plan, int32_t which, ptycho_c32 *dst_dev,
                   ptycho_stream_t stream);
int od2p_set_state(ptycho_plan_t *plan, int32_t which, const ptycho_c32 *src_dev,
                   ptycho_stream_t stream);

/*
 * ST-AGM data-fidelity loss of the whole image and its gradients (sections 2.2
 * and 2.4: G_eps(A u; f) with the gradient of eq. objgrad pulled back through
 * A):  loss = sum_j sum_k g_eps((F(w o S_j u))_k; f_jk),
 *      grad_u = sum_j S_j^T (conj(w) o F^* grad g_j),
 *      grad_w = sum_j conj(S_j u) o F^* grad g_j,
 * gradients in the d/dRe + i d/dIm convention.  u_dev: img_h x img_w;
 * w_dev: m x m; loss_dev: 1 float; grad_u_dev (img_h x img_w) and grad_w_dev
 * (m x m) may be NULL.  One pass over the frames forms each exit wave from u
 * and w, its transform, g and grad g, and the gradient frame h_j = F^* grad
 * g_j; the gradients are then gathered from the h_j.  recompute selects where
 * the h_j live:
 *   1: in the plan's frame scratch, for this call only (no extra memory; a
 *      later call recomputes them);
 *   0: in a plan-owned store of J x m x m complex values (allocated on the
 *      first such call and kept until the plan is destroyed), together with
 *      the loss, for a later call with recompute = 2;
 *   2: no pass over the frames: the loss and the gradients come from the
 *      store, which must hold the frames of the last recompute = 0 call with
 *      the same u_dev and w_dev pointers (and unchanged contents: the library
 *      cannot see writes to them) -- else PTYCHO_ERR_STATE.
 * Storing trades J x m x m x 8 bytes for one pass over the frames in a later
 * gradient (the autograd wrapper stores below a size budget and recomputes
 * above it).  Reductions have a fixed order.  Uses plan scratch: calls on one
 * plan must not overlap.  Errors: INVALID_ARG, STATE, OOM, CUDA.
 */
int stagm_loss_grad(ptycho_plan_t *plan, const ptycho_c32 *u_dev, const ptycho_c32 *w_dev,
                    float *loss_dev, ptycho_c32 *grad_u_dev, ptycho_c32 *grad_w_dev,
                    int32_t recompute, ptycho_stream_t stream);

/*
 * Batches of independent reconstructions (nonblind or blind, any supported
 * probe side, mixed image, probe, scan and subdomain sizes).  One ADMM
 * iteration of all members is one frame-update launch per distinct probe side
 * up to 128 -- a persistent kernel over the (member, frame group) work items --
 * and, for m = 256 members, each member's own wave passes in turn (a 256 x 256
 * frame already spans 16 blocks); the frame updates of different probe sides
 * run as parallel branches of the graph -- and one subdomain-update
 * launch over the tiles of all members (two: slot gathers and, for blind
 * members and members with more than 255 frames over a pixel, frame-list
 * gathers), with each blind member's probe update in between, replayed from a
 * CUDA graph.  Members
 * with m = 64 run the 16 x 4 transform split (ptycho_plan_set_fft kind 2, set
 * by the batch).  Each member computes exactly what od2p_iterate computes on
 * it alone in the same split (bitwise).
 *
 * ptycho_batch_plan: geoms[i], f_devs[i] as for ptycho_plan, i < n; the
 *   members are plans owned by the batch (ptycho_batch_member hands out
 *   borrowed pointers for od2p_init, od2p_merge, od2p_get_state, ...; do not
 *   destroy them, and do not iterate a member on its own between batch
 *   iterations -- the call returns PTYCHO_ERR_STATE).
 * ptycho_batch_iterate: n_iter iterations of every member; od2p_init must
 *   have been called on each.  Errors: INVALID_ARG, UNSUPPORTED, STATE, OOM,
 *   CUDA.
 */
typedef struct ptycho_batch_s ptycho_batch_t;
int ptycho_batch_plan(ptycho_batch_t **out, const ptycho_geometry *geoms, const float *const *f_devs, int32_t n,
                      ptycho_stream_t stream);
int ptycho_batch_destroy(ptycho_batch_t *batch);
int ptycho_batch_size(const ptycho_batch_t *batch, int32_t *n_out);
int ptycho_batch_member(const ptycho_batch_t *batch, int32_t i, ptycho_plan_t **plan_out);
int ptycho_batch_iterate(ptycho_batch_t *batch, int32_t n_iter, ptycho_stream_t stream);
/* Launch shape of the batch's frame updates and of every member's own, as for
 * ptycho_plan_set_launch (one variant and cap for every probe side).         */
int ptycho_batch_set_launch(ptycho_batch_t *batch, int32_t variant, int32_t blocks_per_sm, ptycho_stream_t stream);
int ptycho_batch_get_launch(const ptycho_batch_t *batch, int32_t *variant, int32_t *blocks_per_sm);

/*
 * Allocation-free ST-AGM loss.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- code running while
 * a CUDA stream is being captured into a graph (allocation is not a capturable
 * operation), hosts that hand a plug-in a fixed memory budget, and real-time
 * loops that must not pay cudaMalloc's implicit device synchronisation.  It
 * computes the same value as the `loss` output of stagm_loss_grad, without a
 * plan: sum over frames j and pixels k of g_eps((F(w o S_j u))_k; f_jk).
 *
 * u_dev: img_h x img_w; w_dev: m x m (m in {16, 32, 64, 128});
 * offsets_dev: device int32, n_frames x 2 top-left (row, col), each window
 * inside the image.  They are device memory, so the host cannot check them;
 * the kernel does: a frame whose window leaves the image is not read, and the
 * call then writes NaN to loss_dev;
 * f_dev: n_frames x m x m, natural frequency order; loss_dev: 1 float, written.
 * It allocates nothing.  Its only scratch is a fixed array of 65536 floats
 * (256 KiB) compiled into the library, which every GPU that loads the library
 * holds until the process exits; a call covers at most 65536 thread blocks of
 * frames (65536 frames for m = 64 or 128, 262144 for m = 32, 524288 for
 * m = 16) and returns PTYCHO_ERR_INVALID_ARG beyond that.  The first call on
 * each device looks the array's device address up, and the first call per m
 * raises that kernel's shared-memory limit: make those first calls before any
 * stream capture.  All calls share the one array (each call overwrites every
 * slot it reads, so nothing needs clearing), so calls that overlap on the GPU
 * -- on different streams, or from different threads -- race and must not be
 * issued.  Errors: INVALID_ARG, UNSUPPORTED, CUDA.
 */
int stagm_loss_noalloc(const ptycho_c32 *u_dev, int32_t img_h, int32_t img_w, const ptycho_c32 *w_dev,
                       int32_t m, const int32_t *offsets_dev, int32_t n_frames, const float *f_dev,
                       float eps, float *loss_dev, ptycho_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* OD2P_H */
