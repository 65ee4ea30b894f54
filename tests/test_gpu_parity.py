"""CUDA path vs the FP64 oracle on identical seeded inputs (through the C ABI).

Tolerances (stated in the build's accuracy contract): one iteration within
1e-5 relative L2 per state array; a full run within 1e-3 relative L2 after
global-phase alignment; integer layouts bit-exact; repeated runs bitwise equal.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2011_00162_gb300 as od
from paper_2011_00162_gb300 import synth
from paper_2011_00162_gb300 import build as odbuild

from _cases import make_case, phase_aligned_rel, record, rel_l2

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
ONE_ITER_TOL = 1e-5
END_TOL = 1e-3


def c64(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, np.complex64))).to(DEV)


def f32(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, np.float32))).to(DEV)


def host(t):
    return t.detach().cpu().numpy()


def geom_of(p, offs, **kw):
    d = dict(eps=p.eps, eta=p.eta, r=p.r, mu=p.mu, gamma=p.gamma, blind=p.blind)
    d.update(kw)
    return od.Geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px, **d)


def pair_of(p, offs, w, f, u0=None, **kw):
    g = geom_of(p, offs, **kw)
    plan = od.ptycho_plan(g, f32(f))
    od.od2p_init(plan, c64(w), c64(u0) if u0 is not None else None)
    ref = oracle.ADMM(f, w, offs, p.n, p.n, p.sub_rows, p.sub_cols, p.overlap_px, g.eps, g.eta, g.r,
                      u0=u0, blind=g.blind, mu=g.mu, gamma=g.gamma, mask=g.fourier_support)
    return plan, ref


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    odbuild.build()


# ----------------------------------------------------------------------------- pointwise / operators
@pytest.mark.parametrize("eps,lam", [(0.5, 0.1), (0.5, 5.0), (0.2, 10.0), (0.9, 0.5)])
def test_prox_matches_oracle(eps, lam):
    rng = np.random.default_rng(1)
    n = 200_003  # ragged length
    y = ((rng.standard_normal(n) + 1j * rng.standard_normal(n)) * rng.choice([0.01, 1, 5], n)).astype(np.complex64)
    f = (np.abs(rng.standard_normal(n)) * rng.choice([0, 1, 10], n)).astype(np.float32)
    z = host(od.stagm_prox(c64(y), f32(f), eps, lam))
    ref = oracle.stagm_prox(y, f.astype(np.float64), eps, lam)
    keep = np.abs(y) > 1e-6 * np.sqrt(f)  # sign(0) is arbitrary (any phase is optimal)
    err = np.abs(z - ref)[keep] / (np.abs(ref) + np.sqrt(f) + 1e-30)[keep]
    assert err.max() < 2e-6


@pytest.mark.parametrize("m,n,step,jit", [(16, 61, 5, 1), (32, 100, 9, 2), (64, 300, 16, 2), (128, 400, 40, 3),
                                          (256, 600, 64, 3), (48, 151, 12, 2), (80, 243, 20, 2), (96, 301, 24, 3)])
def test_forward_and_adjoint_match_oracle(m, n, step, jit):
    rng = np.random.default_rng(m)
    offs = synth.raster_offsets(n, m, step, jit, seed=3)
    u = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
    w = synth.make_probe(m)
    f = np.ones((len(offs), m, m), np.float32)
    plan = od.ptycho_plan(od.Geometry(n, n, m, offs), f32(f))
    fr = host(od.ptycho_forward(plan, c64(u), c64(w)))
    ref = oracle.forward(u, w, offs)
    per_frame = np.linalg.norm((fr - ref).reshape(len(offs), -1), axis=1) / np.linalg.norm(ref.reshape(len(offs), -1), axis=1)
    assert per_frame.max() < 1e-6
    y = (rng.standard_normal(ref.shape) + 1j * rng.standard_normal(ref.shape)).astype(np.complex64)
    adj = host(od.overlap_add(plan, c64(y), c64(w), ifft=True))
    assert rel_l2(adj, oracle.adjoint(y, w, offs, n, n)) < 1e-6
    # without the inverse FFT: sum_j S_j^T (conj(w) o y_j), pixels nobody covers are 0
    plain = host(od.overlap_add(plan, c64(y), c64(w), ifft=False))
    exp = np.zeros((n, n), np.complex128)
    for j, (r0, c0) in enumerate(offs):
        exp[r0:r0 + m, c0:c0 + m] += np.conj(w) * y[j]
    assert rel_l2(plain, exp) < 1e-6


@pytest.mark.parametrize("grid,ov,n,m,step,jit", [((1, 2), 8, 64, 16, 4, 0), ((4, 4), 16, 512, 64, 16, 2),
                                                 ((3, 5), 0, 300, 32, 12, 3), ((1, 1), 0, 100, 16, 7, 1),
                                                 ((2, 3), 40, 257, 64, 9, 2)])
def test_decomposition_bit_exact(grid, ov, n, m, step, jit):
    offs = synth.raster_offsets(n, m, step, jit, seed=5)
    plan = od.ptycho_plan(od.Geometry(n, n, m, offs, grid[0], grid[1], ov),
                          f32(np.ones((len(offs), m, m))))
    fs, rect, pr, prc = plan.layout()
    fs_o, rect_o = oracle.geometry(n, n, m, offs, grid[0], grid[1], ov)
    pr_o, prc_o = oracle.pairs(rect_o)
    assert np.array_equal(fs, fs_o) and np.array_equal(rect, rect_o)
    assert np.array_equal(pr, pr_o) and np.array_equal(prc, prc_o)


# ----------------------------------------------------------------------------- one iteration
def _compare_state(plan, ref, tol, blind=False):
    out = {}
    for name, wg, wo in [("u", od.STATE_U, oracle.U), ("Gamma", od.STATE_GAMMA, oracle.GAMMA),
                         ("Lambda", od.STATE_LAMBDA, oracle.LAMBDA)] + (
            [("W_d", od.STATE_WD, oracle.WD), ("Delta", od.STATE_DELTA, oracle.DELTA),
             ("w", od.STATE_W, oracle.W)] if blind else []):
        a, b = host(od.od2p_get_state(plan, wg)), ref.get(wo)
        if b.size == 0:
            continue
        out[name] = rel_l2(a, b)
    bad = {k: v for k, v in out.items() if not v < tol}
    assert not bad, f"relative L2 above {tol}: {bad} (all: {out})"
    return out


def _scramble(plan, ref, seed, blind=False):
    rng = np.random.default_rng(seed)
    for wg, wo, base in [(od.STATE_U, oracle.U, 1.0), (od.STATE_GAMMA, oracle.GAMMA, 0.0),
                         (od.STATE_LAMBDA, oracle.LAMBDA, 0.0)] + (
            [(od.STATE_WD, oracle.WD, None), (od.STATE_DELTA, oracle.DELTA, 0.0)] if blind else []):
        n = ref.get(wo).size
        if n == 0:
            continue
        cur = ref.get(wo)
        if base is None:
            v = cur * (1 + 0.1 * (rng.standard_normal(n) + 1j * rng.standard_normal(n)))
        else:
            scale = 0.2 * (np.abs(cur).mean() + 1e-3) if wo == oracle.GAMMA else 0.2
            v = base + scale * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
        v = v.astype(np.complex64)
        ref.set(wo, v)
        od.od2p_set_state(plan, wg, c64(v))


@pytest.mark.parametrize("scrambled", [False, True])
def test_one_iteration_two_subdomains(scrambled):
    p = synth.small_2sub()
    offs, u_true, w, f = make_case(p)
    plan, ref = pair_of(p, offs, w, f)
    if scrambled:
        _scramble(plan, ref, 3)
    od.od2p_iterate(plan, 1)
    ref.iterate(1)
    out = _compare_state(plan, ref, ONE_ITER_TOL)
    record(f"config1_one_iteration_{'scrambled' if scrambled else 'step0'}", **out)


@pytest.mark.parametrize("scrambled", [False, True])
def test_one_iteration_grid4x4_full_size(scrambled):
    """512^2 image, 841 frames of 64^2, 4x4 subdomains, Poisson 1e4: every array compared."""
    p = synth.grid_4x4()
    offs, u_true, w, f = make_case(p)
    plan, ref = pair_of(p, offs, w, f)
    if scrambled:
        _scramble(plan, ref, 4)
    for it in range(2):
        od.od2p_iterate(plan, 1)
        ref.iterate(1)
        out = _compare_state(plan, ref, ONE_ITER_TOL)
        record(f"config2_one_iteration_{'scrambled' if scrambled else 'step0'}_{it}", **out)
        # re-synchronise so that each comparison measures a single iteration
        for wg, wo in [(od.STATE_U, oracle.U), (od.STATE_GAMMA, oracle.GAMMA), (od.STATE_LAMBDA, oracle.LAMBDA)]:
            od.od2p_set_state(plan, wg, c64(ref.get(wo)))


@pytest.mark.parametrize("m,grid,n,step", [(32, (2, 3), 200, 10), (128, (2, 2), 384, 32), (16, (5, 4), 120, 6),
                                           (256, (2, 2), 512, 64), (48, (2, 2), 200, 12), (80, (2, 3), 320, 20),
                                           (96, (2, 2), 384, 24)])
def test_one_iteration_other_sizes(m, grid, n, step):
    p = synth.Problem("t", n, m, step, 2, grid[0], grid[1], 12, 1e5, 1, eta=0.3, r=0.2, seed=m)
    offs, u_true, w, f = make_case(p)
    plan, ref = pair_of(p, offs, w, f)
    _scramble(plan, ref, 5)
    od.od2p_iterate(plan, 1)
    ref.iterate(1)
    _compare_state(plan, ref, ONE_ITER_TOL)


def test_single_frame_single_subdomain_edge():
    m, n = 64, 64
    offs = np.array([[0, 0]], np.int32)
    w = synth.make_probe(m)
    u = synth.make_image(n, 9)
    f = (np.abs(oracle.forward(u, w, offs)) ** 2).astype(np.float32)
    p = synth.Problem("one", n, m, 1, 0, 1, 1, 0, None, 1)
    plan, ref = pair_of(p, offs, w, f)
    od.od2p_iterate(plan, 2)
    ref.iterate(2)
    _compare_state(plan, ref, ONE_ITER_TOL)


# ----------------------------------------------------------------------------- whole runs
def test_end_of_run_two_subdomains():
    """50 iterations (64^2, 169 frames of 16^2, 2 subdomains, noiseless)."""
    p = synth.small_2sub()
    offs, u_true, w, f = make_case(p)
    plan, ref = pair_of(p, offs, w, f)
    od.od2p_iterate(plan, p.n_iter)
    ref.iterate(p.n_iter)
    ug = host(od.od2p_merge(plan))
    uo = ref.merge()
    lit = synth.lit_mask(p.n, p.n, p.m, offs)
    err = phase_aligned_rel(ug, uo)
    err_truth_oracle = phase_aligned_rel(uo[lit], u_true[lit])
    err_truth_gpu = phase_aligned_rel(ug[lit], u_true[lit])
    print(f"end-of-run GPU vs FP64 oracle {err:.2e}; vs truth: oracle {err_truth_oracle:.3e}, GPU {err_truth_gpu:.3e}")
    record("config1_end_of_run_50its", gpu_vs_oracle=err, oracle_vs_truth=err_truth_oracle,
           gpu_vs_truth=err_truth_gpu)
    assert err < END_TOL
    # after 50 iterations the metrics inherit the trajectory's FP32 deviation: RF (a
    # sum over all frames) within END_TOL, RE (a difference of iterates) within 10 END_TOL
    rf_g, re_g = od.od2p_metrics(plan)
    rf_o, re_o = ref.metrics()
    assert abs(rf_g - rf_o) < END_TOL * rf_o and abs(re_g - re_o) < 10 * END_TOL * re_o


def test_end_of_run_grid4x4():
    """200 iterations of the 512^2 / 841-frame / 4x4 workload."""
    p = synth.grid_4x4()
    offs, u_true, w, f = make_case(p)
    plan, ref = pair_of(p, offs, w, f)
    od.od2p_iterate(plan, p.n_iter)
    ref.iterate(p.n_iter)
    ug, uo = host(od.od2p_merge(plan)), ref.merge()
    lit = synth.lit_mask(p.n, p.n, p.m, offs)
    err = phase_aligned_rel(ug, uo)
    err_truth_oracle = phase_aligned_rel(uo[lit], u_true[lit])
    print(f"end-of-run GPU vs FP64 oracle {err:.2e}; oracle vs truth {err_truth_oracle:.3e}")
    record("config2_end_of_run_200its", gpu_vs_oracle=err, oracle_vs_truth=err_truth_oracle,
           gpu_vs_truth=phase_aligned_rel(ug[lit], u_true[lit]))
    assert err < END_TOL


def test_bitwise_determinism_and_graph_equals_stages():
    p = synth.grid_4x4()
    offs, u_true, w, f = make_case(p)
    outs = []
    for mode in ("graph", "graph", "stages"):
        plan = od.ptycho_plan(geom_of(p, offs), f32(f))
        od.od2p_init(plan, c64(w))
        for _ in range(3):
            if mode == "graph":
                od.od2p_iterate(plan, 1)
            else:
                od.od2p_frame_update(plan)
                od.od2p_subdomain_update(plan)
        outs.append([host(od.od2p_get_state(plan, k)) for k in (od.STATE_U, od.STATE_GAMMA, od.STATE_LAMBDA)])
        plan.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    for a, b in zip(outs[0], outs[2]):
        assert np.array_equal(a, b)


def test_blind_graph_equals_stages():
    """A blind iteration replayed from its graph equals frame update, probe
    update and subdomain update called one by one, bit for bit."""
    q = synth.Problem("bstage", 96, 32, 6, 1, 2, 2, 8, None, 1, eta=0.5, r=0.1, blind=True, mu=1.0, seed=4)
    offs, u_true, w, f = make_case(q)
    keys = (od.STATE_U, od.STATE_GAMMA, od.STATE_LAMBDA, od.STATE_WD, od.STATE_DELTA, od.STATE_W)
    outs = []
    for mode in ("graph", "stages"):
        plan = od.ptycho_plan(geom_of(q, offs), f32(f))
        od.od2p_init(plan, c64(synth.gaussian_probe(q.m)))
        for _ in range(3):
            if mode == "graph":
                od.od2p_iterate(plan, 1)
            else:
                od.od2p_frame_update(plan)
                od.probe_update(plan)
                od.od2p_subdomain_update(plan)
        outs.append([host(od.od2p_get_state(plan, k)) for k in keys])
        plan.close()
    for k, a, b in zip(keys, *outs):
        assert np.array_equal(a, b), k


def test_metrics_and_merge_match_oracle():
    p = synth.grid_4x4()
    offs, u_true, w, f = make_case(p)
    plan, ref = pair_of(p, offs, w, f)
    od.od2p_iterate(plan, 3)
    ref.iterate(3)
    rf_g, re_g = od.od2p_metrics(plan)
    rf_o, re_o = ref.metrics()
    assert abs(rf_g - rf_o) < 1e-5 * rf_o and abs(re_g - re_o) < 1e-4 * re_o
    assert rel_l2(host(od.od2p_merge(plan)), ref.merge()) < ONE_ITER_TOL


def _oracle_subdomain_loss(ref, f, offs, p):
    """sum_d sum_{j in d} G_eps(F(W_d o S_j u_d); f_j) with the oracle's loss,
    each subdomain copy u_d taken as an image of its rectangle."""
    fs, rect = oracle.geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px)
    u = ref.get(oracle.U)
    Wd = ref.get(oracle.WD).reshape(len(rect), p.m, p.m)
    total, k = 0.0, 0
    for d, (r0, c0, r1, c1) in enumerate(rect):
        n = (r1 - r0) * (c1 - c0)
        ud = u[k:k + n].reshape(r1 - r0, c1 - c0)
        k += n
        sel = np.flatnonzero(fs == d)
        if len(sel):
            loc = offs[sel] - np.array([r0, c0], np.int32)
            total += oracle.loss_grad(ud, Wd[d], loc, np.asarray(f, np.float64)[sel], p.eps)[0]
    return total


@pytest.mark.parametrize("blind,m", [(False, 64), (True, 32), (False, 48), (True, 256), (False, 128)])
def test_metrics_loss_matches_oracle(blind, m):
    """od2p_metrics' loss: the ST-AGM data term of the current subdomain iterate."""
    n = {32: 96, 48: 144, 64: 256, 128: 384, 256: 512}[m]
    p = synth.Problem("ml", n, m, m // 4, 1, 2, 2, 8, 1e4, 1, eta=2.0, r=0.5, blind=blind,
                      mu=1.0 if blind else 0.0, gamma=0.1 if blind else 0.0, seed=31)
    offs, u_true, w, f = make_case(p)
    w0 = synth.gaussian_probe(m) if blind else w
    plan, ref = pair_of(p, offs, w0, f)
    od.od2p_iterate(plan, 2)
    ref.iterate(2)
    rf, re, loss = od.od2p_metrics(plan, loss=True)
    exp = _oracle_subdomain_loss(ref, f, offs, p)
    assert abs(loss - exp) <= ONE_ITER_TOL * abs(exp), (loss, exp)
    record(f"metrics_loss_m{m}_{'blind' if blind else 'nonblind'}", loss_rel=abs(loss - exp) / abs(exp))
    # the extra pass leaves the state and the other metrics alone
    u0 = od.od2p_get_state(plan, od.STATE_U).clone()
    assert od.od2p_metrics(plan) == (rf, re)
    assert torch.equal(od.od2p_get_state(plan, od.STATE_U), u0)


def test_checkpoint_resume_bitwise():
    p = synth.small_2sub()
    offs, u_true, w, f = make_case(p)
    a = od.ptycho_plan(geom_of(p, offs), f32(f))
    od.od2p_init(a, c64(w))
    od.od2p_iterate(a, 10)
    snap = {k: od.od2p_get_state(a, k).clone() for k in (od.STATE_U, od.STATE_GAMMA, od.STATE_LAMBDA)}
    od.od2p_iterate(a, 10)
    b = od.ptycho_plan(geom_of(p, offs), f32(f))
    od.od2p_init(b, c64(w))
    for k, v in snap.items():
        od.od2p_set_state(b, k, v)
    od.od2p_iterate(b, 10)
    for k in snap:
        assert torch.equal(od.od2p_get_state(a, k), od.od2p_get_state(b, k))


# ----------------------------------------------------------------------------- blind
@pytest.mark.parametrize("masked,m,n,step", [(False, 32, 96, 8), (True, 32, 96, 8), (False, 256, 512, 64),
                                             (True, 256, 512, 64), (False, 48, 144, 12), (True, 96, 288, 24)])
def test_blind_one_iteration(masked, m, n, step):
    p = synth.Problem("b", n, m, step, 1, 2, 2, 8, 1e5, 1, eta=0.3, r=0.2, blind=True, mu=2.0,
                      gamma=0.1, seed=21)
    offs, u_true, w_true, f = make_case(p)
    w0 = synth.gaussian_probe(p.m)
    mask = None
    if masked:
        yy, xx = np.meshgrid(np.fft.fftfreq(p.m), np.fft.fftfreq(p.m), indexing="ij")
        mask = (np.hypot(yy, xx) < 0.3).astype(np.uint8)
    g = geom_of(p, offs, fourier_support=mask)
    plan = od.ptycho_plan(g, f32(f))
    od.od2p_init(plan, c64(w0))
    ref = oracle.ADMM(f, w0, offs, p.n, p.n, p.sub_rows, p.sub_cols, p.overlap_px, p.eps, p.eta, p.r,
                      blind=True, mu=p.mu, gamma=p.gamma, mask=mask)
    _scramble(plan, ref, 8, blind=True)
    for _ in range(2):
        od.od2p_iterate(plan, 1)
        ref.iterate(1)
        _compare_state(plan, ref, ONE_ITER_TOL, blind=True)
        for wg, wo in [(od.STATE_U, oracle.U), (od.STATE_GAMMA, oracle.GAMMA), (od.STATE_LAMBDA, oracle.LAMBDA),
                       (od.STATE_WD, oracle.WD), (od.STATE_DELTA, oracle.DELTA), (od.STATE_W, oracle.W)]:
            od.od2p_set_state(plan, wg, c64(ref.get(wo)))


# ----------------------------------------------------------------------------- loss and gradients
@pytest.mark.parametrize("m,n,step", [(16, 64, 4), (64, 256, 16), (128, 384, 48), (256, 512, 96), (48, 192, 12),
                                      (80, 240, 20), (96, 288, 24)])
def test_loss_and_gradients_match_oracle(m, n, step):
    p = synth.Problem("g", n, m, step, 2, 1, 1, 0, 1e4, 1, seed=m + 1)
    offs, u_true, w, f = make_case(p)
    rng = np.random.default_rng(2)
    u = (u_true * (1 + 0.2 * (rng.standard_normal(u_true.shape) + 1j * rng.standard_normal(u_true.shape)))).astype(np.complex64)
    wp = (w * (1 + 0.1 * rng.standard_normal(w.shape))).astype(np.complex64)
    plan = od.ptycho_plan(od.Geometry(n, n, m, offs, eps=0.5), f32(f))
    loss, gu, gw = od.stagm_loss_grad(plan, c64(u), c64(wp))
    L, gu_o, gw_o = oracle.loss_grad(u, wp, offs, f.astype(np.float64), 0.5)
    assert abs(float(loss.item()) - L) < 1e-5 * abs(L)
    assert rel_l2(host(gu), gu_o) < 1e-5
    assert rel_l2(host(gw), gw_o) < 1e-5


# ----------------------------------------------------------------------------- full-size m = 256
def test_large_blind_workload_sampled_frames():
    """4096^2 image, 6561 frames of 256^2, 8x8 subdomains: one frame update on the
    GPU, and the updated Gamma_j and residual q_j of sampled frames recomputed
    frame by frame by the oracle (forward, prox, inverse)."""
    p = synth.large_blind()
    offs = p.offsets()
    assert len(offs) == 6561
    u_true, w_true = p.truth(), p.probe()
    f = synth.poissonize(np.abs(oracle.forward(u_true, w_true, offs)) ** 2, p.peak, 11)
    w0 = synth.gaussian_probe(p.m)
    eta = 2.0
    g = od.Geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px, eps=0.5, eta=eta, r=0.5,
                    mu=1.0, gamma=0.0, blind=True)
    plan = od.ptycho_plan(g, f32(f))
    rng = np.random.default_rng(6)
    u0 = (u_true * (1 + 0.1 * rng.standard_normal(u_true.shape))).astype(np.complex64)
    od.od2p_init(plan, c64(w0), c64(u0))
    od.od2p_frame_update(plan)
    gam = od.od2p_get_state(plan, od.STATE_GAMMA)
    q = od.od2p_get_state(plan, od.STATE_Q)
    mm = p.m * p.m
    worst = [0.0, 0.0]
    for j in rng.choice(len(offs), 12, replace=False):
        r0, c0 = offs[j]
        x = oracle.forward(u0, w0, offs[j:j + 1])[0]          # A u for frame j (u_d = R_d u0)
        z = oracle.stagm_prox(x, f[j].astype(np.float64), 0.5, eta)
        g_ref = x - z                                          # Gamma^0 = 0
        q_ref = oracle.fft2(z - g_ref, True)
        eg, eq = rel_l2(host(gam[j * mm:(j + 1) * mm]), g_ref), rel_l2(host(q[j * mm:(j + 1) * mm]), q_ref)
        worst = [max(worst[0], eg), max(worst[1], eq)]
        assert eg < ONE_ITER_TOL
        assert eq < ONE_ITER_TOL
    record("config5_sampled_frames_one_update", Gamma=worst[0], q=worst[1])


def test_nonblind_residual_frames_from_gather_slots():
    """q_j = conj(w) o F^*(z_j - Gamma_j) exported from the nonblind gather slots."""
    p = synth.grid_4x4()
    offs, u_true, w, f = make_case(p)
    plan, ref = pair_of(p, offs, w, f)
    _scramble(plan, ref, 9)
    od.od2p_iterate(plan, 1)
    ref.iterate(1)
    mm = p.m * p.m
    z, gam = ref.get(oracle.Z).reshape(-1, p.m, p.m), ref.get(oracle.GAMMA).reshape(-1, p.m, p.m)
    q = host(od.od2p_get_state(plan, od.STATE_Q)).reshape(-1, p.m, p.m)
    for j in np.random.default_rng(1).choice(len(offs), 20, replace=False):
        q_ref = np.conj(w) * oracle.fft2(z[j] - gam[j], True)
        assert rel_l2(q[j], q_ref) < ONE_ITER_TOL


def test_blind_workload_1024_full_size():
    """1024^2 image, 841 frames of 128^2, 4x4 subdomains, Gaussian initial probe,
    Poisson 1e4: one blind iteration (Algorithm 3) from a scrambled state, every
    state array compared; then the ST-AGM loss and both gradients at full size."""
    p = synth.blind_4x4()
    offs, u_true, w_true, f = make_case(p)
    assert len(offs) == 841
    w0 = synth.gaussian_probe(p.m)
    eta, r, mu, gamma = 2.0, 0.5, 1.0, 0.1
    g = od.Geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px, eps=0.5, eta=eta, r=r, mu=mu,
                    gamma=gamma, blind=True)
    plan = od.ptycho_plan(g, f32(f))
    od.od2p_init(plan, c64(w0))
    ref = oracle.ADMM(f, w0, offs, p.n, p.n, p.sub_rows, p.sub_cols, p.overlap_px, 0.5, eta, r, blind=True,
                      mu=mu, gamma=gamma)
    _scramble(plan, ref, 12, blind=True)
    od.od2p_iterate(plan, 1)
    ref.iterate(1)
    out = _compare_state(plan, ref, ONE_ITER_TOL, blind=True)
    record("config4_one_iteration_scrambled", **out)
    rng = np.random.default_rng(3)
    u = (u_true * (1 + 0.1 * rng.standard_normal(u_true.shape))).astype(np.complex64)
    loss, gu, gw = od.stagm_loss_grad(plan, c64(u), c64(w0))
    L, gu_o, gw_o = oracle.loss_grad(u, w0, offs, f.astype(np.float64), 0.5)
    record("config4_loss_grad", loss=abs(float(loss.item()) - L) / abs(L), grad_u=rel_l2(host(gu), gu_o),
           grad_w=rel_l2(host(gw), gw_o))
    assert abs(float(loss.item()) - L) < 1e-5 * abs(L)
    assert rel_l2(host(gu), gu_o) < 1e-5 and rel_l2(host(gw), gw_o) < 1e-5


@pytest.mark.parametrize("m,n,step", [(16, 64, 4), (32, 100, 9), (64, 300, 16), (128, 384, 48), (256, 512, 96),
                                      (48, 144, 12), (80, 240, 20), (96, 288, 24)])
def test_probe_init_matches_oracle(m, n, step):
    """Section 4.2's data-driven initial probe from a plan's intensities."""
    p = synth.Problem("pi", n, m, step, 1, 2, 2, 8, 1e4, 1, seed=m)
    offs, u_true, w, f = make_case(p)
    plan = od.ptycho_plan(geom_of(p, offs), f32(f))
    w0 = host(od.ptycho_probe_init(plan))
    ref = oracle.probe_init(f.astype(np.float64))
    err = rel_l2(w0, ref)
    record(f"probe_init_m{m}", w0=err)
    assert err < ONE_ITER_TOL
    # a probe whose spectrum is real and positive is recovered exactly (up to FP32)
    rng = np.random.default_rng(m)
    a = (0.1 + rng.random((m, m))).astype(np.float32)
    fa = np.repeat((a.astype(np.float64) ** 2)[None], len(offs), axis=0).astype(np.float32)
    plan2 = od.ptycho_plan(geom_of(p, offs), f32(fa))
    assert rel_l2(host(od.ptycho_probe_init(plan2)), np.fft.ifft2(a.astype(np.float64), norm="ortho")) < ONE_ITER_TOL


def test_plans_reuse_pooled_memory_bitwise():
    """Plans take device memory from a pool that keeps what destroyed plans free;
    a plan built on reused (dirty) memory computes exactly what a fresh one does."""
    p = synth.grid_4x4()
    offs, u_true, w, f = make_case(p)
    outs = []
    for k in range(3):
        if k == 2:
            od.ptycho_release_cached_memory()
        plan = od.ptycho_plan(geom_of(p, offs), f32(f))
        od.od2p_init(plan, c64(w))
        od.od2p_iterate(plan, 3)
        outs.append([host(od.od2p_get_state(plan, s)) for s in (od.STATE_U, od.STATE_GAMMA, od.STATE_LAMBDA)])
        # scribble over the plan's memory before it goes back to the pool
        od.od2p_set_state(plan, od.STATE_GAMMA, torch.full((od.od2p_state_len(plan, od.STATE_GAMMA),), 7 + 7j,
                                                           dtype=torch.complex64, device=DEV))
        plan.close()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


def test_dense_scan_takes_the_list_gather():
    """More than 255 frames over a pixel (m = 32, step 2: up to 256): the
    nonblind plan gathers through frame lists with the known probe; one
    iteration from a scrambled state and the exported residual still match the
    oracle, and a batch member with such a scan equals its plan alone."""
    # one subdomain: its frames are all frames (coverage is counted per subdomain)
    p = synth.Problem("dense", 80, 32, 2, 0, 1, 1, 0, 1e5, 1, eta=0.3, r=0.2, seed=4)
    offs, u_true, w, f = make_case(p)
    cover = np.zeros((p.n, p.n), int)
    for r0, c0 in offs:
        cover[r0:r0 + p.m, c0:c0 + p.m] += 1
    assert cover.max() > 255
    plan, ref = pair_of(p, offs, w, f)
    _scramble(plan, ref, 5)
    od.od2p_iterate(plan, 1)
    ref.iterate(1)
    out = _compare_state(plan, ref, ONE_ITER_TOL)
    record("dense_scan_list_gather_one_iteration", **out)
    z, gam = ref.get(oracle.Z).reshape(-1, p.m, p.m), ref.get(oracle.GAMMA).reshape(-1, p.m, p.m)
    q = host(od.od2p_get_state(plan, od.STATE_Q)).reshape(-1, p.m, p.m)
    for j in np.random.default_rng(2).choice(len(offs), 10, replace=False):
        assert rel_l2(q[j], np.conj(w) * oracle.fft2(z[j] - gam[j], True)) < ONE_ITER_TOL
    # a batch takes such a member: one iteration from the same start equals the plan alone
    batch = od.ptycho_batch_plan([geom_of(p, offs)], [f32(f)])
    alone = od.ptycho_plan(geom_of(p, offs), f32(f))
    for pl in (batch.members[0], alone):
        od.od2p_init(pl, c64(w))
    batch.iterate(1)
    od.od2p_iterate(alone, 1)
    for k in (od.STATE_U, od.STATE_GAMMA, od.STATE_LAMBDA):
        assert torch.equal(od.od2p_get_state(batch.members[0], k), od.od2p_get_state(alone, k)), k
    batch.close()
    alone.close()


def test_blind_checkpoint_resume_bitwise():
    """Every blind state (u, Gamma, Lambda, W_d, Delta, w) exported after 6
    iterations and loaded into a fresh plan continues bit for bit."""
    p = synth.Problem("bres", 96, 32, 8, 1, 2, 2, 8, 1e5, 1, eta=2.0, r=0.5, blind=True, mu=1.0, gamma=0.1, seed=3)
    offs, u_true, w, f = make_case(p)
    w0 = synth.gaussian_probe(p.m)
    a = od.ptycho_plan(geom_of(p, offs), f32(f))
    od.od2p_init(a, c64(w0))
    od.od2p_iterate(a, 6)
    keys = (od.STATE_U, od.STATE_GAMMA, od.STATE_LAMBDA, od.STATE_WD, od.STATE_DELTA, od.STATE_W)
    snap = {k: od.od2p_get_state(a, k).clone() for k in keys}
    od.od2p_iterate(a, 5)
    b = od.ptycho_plan(geom_of(p, offs), f32(f))
    od.od2p_init(b, c64(w0))
    for k, v in snap.items():
        od.od2p_set_state(b, k, v)
    od.od2p_iterate(b, 5)
    for k in keys:
        assert torch.equal(od.od2p_get_state(a, k), od.od2p_get_state(b, k)), k


def test_reconstructions_converge():
    """The method does what the paper says: noiseless nonblind data (2 subdomains)
    reach the truth up to a global phase, and a blind run from a Gaussian probe
    drives RF down by an order of magnitude."""
    p = synth.small_2sub()
    offs, u_true, w, f = make_case(p)
    plan = od.ptycho_plan(geom_of(p, offs), f32(f))  # the paper's eta = 0.1, r = 0.05
    od.od2p_init(plan, c64(w))
    od.od2p_iterate(plan, 300)
    lit = synth.lit_mask(p.n, p.n, p.m, offs)
    err = phase_aligned_rel(host(od.od2p_merge(plan))[lit], u_true[lit])
    rf, re = od.od2p_metrics(plan)
    record("convergence_nonblind_300its", err_vs_truth=err, rf=rf)
    assert err < 1e-3 and rf < 1e-3, (err, rf)  # the FP64 oracle reaches 3e-7 and 4e-8
    q = synth.Problem("bconv", 96, 32, 6, 1, 2, 2, 8, None, 1, eta=0.5, r=0.1, blind=True, mu=1.0, seed=4)
    offs, u_true, w, f = make_case(q)
    bp = od.ptycho_plan(geom_of(q, offs), f32(f))
    od.od2p_init(bp, c64(synth.gaussian_probe(q.m)))
    od.od2p_iterate(bp, 5)
    rf0, _ = od.od2p_metrics(bp)
    od.od2p_iterate(bp, 300)
    rf1, _ = od.od2p_metrics(bp)
    record("convergence_blind_300its", rf_start=rf0, rf_end=rf1)
    assert rf1 < 0.1 * rf0, (rf0, rf1)


def test_snr_matches_oracle():
    """od2p_snr equals section 4's SNR computed in FP64 from the GPU's own merged
    image (all pixels, and the illuminated ones), and the closed form for a
    recovery that is the truth scaled by 1.1 and phase-rotated."""
    p = synth.small_2sub()
    offs, u_true, w, f = make_case(p)
    plan = od.ptycho_plan(geom_of(p, offs), f32(f))
    od.od2p_init(plan, c64(w))
    od.od2p_iterate(plan, 20)
    ug = host(od.od2p_merge(plan))
    lit = synth.lit_mask(p.n, p.n, p.m, offs)
    got = od.od2p_snr(plan, c64(u_true))
    got_lit = od.od2p_snr(plan, c64(u_true), torch.from_numpy(lit).to(DEV))
    want, want_lit = oracle.snr(ug, u_true), oracle.snr(ug[lit], u_true[lit])
    record("snr_20its", gpu=got, oracle=want, gpu_lit=got_lit, oracle_lit=want_lit)
    assert abs(got - want) < 1e-3 * max(1.0, abs(want)), (got, want)
    assert abs(got_lit - want_lit) < 1e-3 * max(1.0, abs(want_lit)), (got_lit, want_lit)
    # u_r = 1.1 e^{0.7i} u_g everywhere: SNR = 20 + 10 log10(1.21) dB
    t = (1.1 * np.exp(0.7j) * u_true).astype(np.complex64)
    _, rect, _, _ = plan.layout()  # copies stored subdomain after subdomain, row-major
    u = np.concatenate([t[r0:r1, c0:c1].reshape(-1) for r0, c0, r1, c1 in rect])
    od.od2p_set_state(plan, od.STATE_U, c64(u))
    assert abs(od.od2p_snr(plan, c64(u_true)) - (20.0 + 10 * np.log10(1.21))) < 1e-3


def test_peak_probes_compute_what_they_claim():
    """The ceiling probes do their arithmetic: the FMA chains follow the closed
    form x_n = a^n x_0 + b (1 - a^n) / (1 - a); the shared-memory probe's sums are
    exact small integers."""
    nb, iters = 3, 10
    sink = torch.empty(nb * 256, dtype=torch.float32, device=DEV)
    od.ptycho_peak_probe(od.PROBE_FMA, nb, iters, sink)
    a, b = 0.999999, 1e-7
    t = np.arange(256)
    want = sum(a ** iters * (t + i) + b * (1 - a ** iters) / (1 - a) for i in range(8))
    got = host(sink).reshape(nb, 256)
    assert np.allclose(got, want[None, :], rtol=1e-5)
    od.ptycho_peak_probe(od.PROBE_SMEM, nb, iters, sink)
    lane, warp = t % 32, t // 32
    want = sum(((warp * 8 + i + k) & 63) * 32 + lane for k in range(iters) for i in range(8)) + iters * 8 * 6
    assert np.array_equal(host(sink).reshape(nb, 256), np.broadcast_to(want.astype(np.float32), (nb, 256)))


@pytest.mark.parametrize("blind", [False, True])
def test_iterate_until_equals_host_stopping_loop(blind):
    """The device-side stopping loop stops after the same iteration as a host
    loop that reads RF after every iteration, with bitwise-equal state, for an
    odd and an even stopping point and at the iteration cap; iterating on from
    its end continues the same trajectory."""
    if blind:
        q = synth.Problem("buntil", 96, 32, 6, 1, 2, 2, 8, None, 1, eta=0.5, r=0.1, blind=True, mu=1.0, seed=4)
        offs, u_true, w, f = make_case(q)
        w0 = synth.gaussian_probe(q.m)
    else:
        q = synth.small_2sub()
        offs, u_true, w, f = make_case(q)
        w0 = w
    keys = (od.STATE_U, od.STATE_GAMMA, od.STATE_LAMBDA) + ((od.STATE_WD, od.STATE_W) if blind else ())

    def fresh():
        plan = od.ptycho_plan(geom_of(q, offs), f32(f))
        od.od2p_init(plan, c64(w0))
        return plan

    ref = fresh()
    rfs, snaps = [], []
    for _ in range(14):
        od.od2p_iterate(ref, 1)
        rfs.append(np.float32(od.od2p_metrics(ref)[0]))
        snaps.append([host(od.od2p_get_state(ref, k)) for k in keys])
    for k_stop in (7, 10):  # odd and even iteration counts
        tol = float(rfs[k_stop - 1])
        want = next(i + 1 for i, v in enumerate(rfs) if v <= np.float32(tol))
        plan = fresh()
        n, rf = od.od2p_iterate_until(plan, tol, 100)
        assert n == want and np.float32(rf) == rfs[n - 1], (n, want, rf, rfs[n - 1])
        for k, a in zip(keys, snaps[n - 1]):
            assert np.array_equal(host(od.od2p_get_state(plan, k)), a), k
        od.od2p_iterate(plan, 14 - n)  # the buffers' parity is carried on
        for k, a in zip(keys, snaps[13]):
            assert np.array_equal(host(od.od2p_get_state(plan, k)), a), k
        plan.close()
    plan = fresh()
    n, rf = od.od2p_iterate_until(plan, 0.0, 5)  # the cap
    assert n == 5 and np.float32(rf) == rfs[4]
    assert od.od2p_iterate_until(plan, 1.0, 0) == (0, 0.0)
    n, _ = od.od2p_iterate_until(plan, 1e9, 50)  # met at once: one iteration runs
    assert n == 1
    for k, a in zip(keys, snaps[5]):
        assert np.array_equal(host(od.od2p_get_state(plan, k)), a), k


def test_concurrent_plans_on_two_streams_and_threads():
    """Two plans driven at once from two host threads on two CUDA streams
    (graph capture, replay, metrics) end bitwise equal to the same plans run one
    after the other."""
    import threading
    cases = [synth.small_2sub(), synth.Problem("conc", 128, 32, 8, 1, 2, 2, 8, 1e4, 1, eta=2.0, r=0.5, seed=9)]
    inputs = [make_case(p) for p in cases]

    def run(i, stream, out):
        p = cases[i]
        offs, _, w, f = inputs[i]
        with torch.cuda.stream(stream):
            plan = od.ptycho_plan(geom_of(p, offs), f32(f), stream=stream)
            od.od2p_init(plan, c64(w), stream=stream)
            for _ in range(5):
                od.od2p_iterate(plan, 4, stream=stream)
                od.od2p_metrics(plan, stream=stream)
            out[i] = [host(od.od2p_get_state(plan, k, stream=stream)) for k in (od.STATE_U, od.STATE_GAMMA)]
            plan.close()

    seq, par = {}, {}
    for i in range(2):
        run(i, torch.cuda.current_stream(), seq)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    th = [threading.Thread(target=run, args=(i, streams[i], par)) for i in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    torch.cuda.synchronize()
    for i in range(2):
        for a, b in zip(seq[i], par[i]):
            assert np.array_equal(a, b), i


@pytest.mark.parametrize("kind", [1, 2])
def test_fft_16x4_frame_update_matches_oracle(kind):
    """The 16 x 4 transform split for m = 64 (ptycho_plan_set_fft): one iteration
    of the full 512^2 / 841-frame / 4x4 workload from a scrambled state, nonblind
    (gather slots) and blind (frame-order residual), every array within the
    one-iteration bar; its own iterates are deterministic and the graph equals
    the stages."""
    p = synth.grid_4x4()
    offs, u_true, w, f = make_case(p)
    plan, ref = pair_of(p, offs, w, f)
    od.ptycho_plan_set_fft(plan, kind)
    assert od.ptycho_plan_get_fft(plan) == kind
    _scramble(plan, ref, 4)
    for it in range(2):
        od.od2p_iterate(plan, 1)
        ref.iterate(1)
        out = _compare_state(plan, ref, ONE_ITER_TOL)
        record(f"config2_fft16x4_kind{kind}_{it}", **out)
        for wg, wo in [(od.STATE_U, oracle.U), (od.STATE_GAMMA, oracle.GAMMA), (od.STATE_LAMBDA, oracle.LAMBDA)]:
            od.od2p_set_state(plan, wg, c64(ref.get(wo)))
    rf, _ = od.od2p_metrics(plan)
    assert abs(rf - ref.metrics()[0]) < 1e-5 * ref.metrics()[0] + 1e-7
    # determinism and graph == stages for this kind
    outs = []
    for mode in ("graph", "graph", "stages"):
        a = od.ptycho_plan(geom_of(p, offs), f32(f))
        od.ptycho_plan_set_fft(a, kind)
        od.od2p_init(a, c64(w))
        for _ in range(3):
            if mode == "graph":
                od.od2p_iterate(a, 1)
            else:
                od.od2p_frame_update(a)
                od.od2p_subdomain_update(a)
        outs.append([host(od.od2p_get_state(a, k)) for k in (od.STATE_U, od.STATE_GAMMA, od.STATE_LAMBDA)])
        a.close()
    for x, y in zip(outs[0], outs[1]):
        assert np.array_equal(x, y)
    for x, y in zip(outs[0], outs[2]):
        assert np.array_equal(x, y)
    # blind: the unweighted residual in frame order
    q = synth.Problem("b64", 256, 64, 16, 1, 2, 2, 8, 1e5, 1, eta=0.3, r=0.2, blind=True, mu=2.0, gamma=0.1,
                      seed=21)
    offs, u_true, w_true, f = make_case(q)
    w0 = synth.gaussian_probe(q.m)
    bp = od.ptycho_plan(geom_of(q, offs), f32(f))
    od.ptycho_plan_set_fft(bp, kind)
    od.od2p_init(bp, c64(w0))
    bref = oracle.ADMM(f, w0, offs, q.n, q.n, q.sub_rows, q.sub_cols, q.overlap_px, q.eps, q.eta, q.r,
                       blind=True, mu=q.mu, gamma=q.gamma)
    _scramble(bp, bref, 8, blind=True)
    od.od2p_iterate(bp, 1)
    bref.iterate(1)
    _compare_state(bp, bref, ONE_ITER_TOL, blind=True)


def test_fft_kind_arguments():
    p = synth.small_2sub()  # m = 16
    offs, u_true, w, f = make_case(p)
    plan = od.ptycho_plan(geom_of(p, offs), f32(f))
    with pytest.raises(RuntimeError):
        od.ptycho_plan_set_fft(plan, 1)
    with pytest.raises(RuntimeError):
        od.ptycho_plan_set_fft(plan, 3)
    od.ptycho_plan_set_fft(plan, 0)
    assert od.ptycho_plan_get_fft(plan) == 0
