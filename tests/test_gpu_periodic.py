"""Periodic boundaries on the GPU against the FP64 oracle's periodic variant
(the torus reading of section 4's periodic boundary): the decomposition with
its shifted pairs and self-pairs, one iteration from a scrambled state, a run
from u = 1, Step 0 modulo the image, the merge, the SNR and the consensus
residual; the image-space operators; the reduction to the vacuum boundary
(shards of a periodic plan: tests/test_gpu_shard.py)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2011_00162_gb300 as od
from paper_2011_00162_gb300 import build as odbuild

from _cases import record, rel_l2

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    odbuild.build()


def _torus_case(H, m, step, jitter, seed, noise=0.05):
    rng = np.random.default_rng(seed)
    offs = np.array([(r, c) for r in range(0, H, step) for c in range(0, H, step)], np.int32)
    offs = ((offs + rng.integers(-jitter, jitter + 1, offs.shape)) % H).astype(np.int32)
    u = (0.5 + 0.5 * rng.random((H, H))) * np.exp(1j * rng.uniform(-1, 1, (H, H)))
    w = (0.5 + rng.random((m, m))) * np.exp(1j * rng.uniform(-2, 2, (m, m)))
    fr = np.stack([np.fft.fft2(w * np.roll(u, (-r, -c), axis=(0, 1))[:m, :m], norm="ortho") for r, c in offs])
    f = np.abs(fr) ** 2 * (1 + noise * rng.random(fr.shape))
    return offs, u, w, f


def _pair(H, m, offs, w, f, grid, ov, blind=False, u0=None, eta=0.3, r=0.2):
    kw = dict(mu=1.0 if blind else 0.0, gamma=0.2 if blind else 0.0, blind=blind)
    g = od.Geometry(H, H, m, offs, grid[0], grid[1], ov, 0.5, eta, r, periodic=True, **kw)
    plan = od.ptycho_plan(g, torch.from_numpy(np.asarray(f, np.float32)).to(DEV))
    w0 = np.asarray(w, np.complex64)
    od.od2p_init(plan, torch.from_numpy(w0).to(DEV),
                 torch.from_numpy(np.asarray(u0, np.complex64)).to(DEV) if u0 is not None else None)
    ref = oracle.ADMM(f, w0, offs, H, H, grid[0], grid[1], ov, 0.5, eta, r, u0=u0, periodic=True, **kw)
    return plan, ref


def _scramble(plan, ref, seed, blind):
    rng = np.random.default_rng(seed)
    sel = [(od.STATE_U, oracle.U), (od.STATE_GAMMA, oracle.GAMMA), (od.STATE_LAMBDA, oracle.LAMBDA)]
    if blind:
        sel += [(od.STATE_WD, oracle.WD), (od.STATE_DELTA, oracle.DELTA)]
    for k, ko in sel:
        n = od.od2p_state_len(plan, k)
        scale = 1.0 if k in (od.STATE_U, od.STATE_WD) else 0.1
        v = ((rng.standard_normal(n) + 1j * rng.standard_normal(n)) * scale).astype(np.complex64)
        if k == od.STATE_U:
            v += 1.0
        od.od2p_set_state(plan, k, torch.from_numpy(v).to(DEV))
        ref.set(ko, v.astype(np.complex128))


def _compare(plan, ref, blind, tol=TOL):
    out = {}
    sel = [(od.STATE_U, oracle.U), (od.STATE_GAMMA, oracle.GAMMA), (od.STATE_LAMBDA, oracle.LAMBDA)]
    if blind:
        sel += [(od.STATE_WD, oracle.WD), (od.STATE_DELTA, oracle.DELTA), (od.STATE_W, oracle.W)]
    for k, ko in sel:
        b = ref.get(ko)
        if b.size:
            out[str(k)] = rel_l2(od.od2p_get_state(plan, k).cpu().numpy(), b)
            assert out[str(k)] < tol, (k, out[str(k)])
    return out


CASES = [(96, 16, 6, 1, (3, 3), 8), (128, 32, 8, 2, (2, 2), 8), (64, 16, 4, 1, (1, 1), 4), (192, 64, 16, 2, (2, 3), 16),
         (512, 256, 64, 4, (2, 2), 32)]


@pytest.mark.parametrize("case", CASES, ids=[f"m{c[1]}_{c[4][0]}x{c[4][1]}" for c in CASES])
def test_periodic_layout_matches_the_oracle(case):
    H, m, step, jit, grid, ov = case
    offs, u, w, f = _torus_case(H, m, step, jit, seed=H + m)
    plan, ref = _pair(H, m, offs, w, f, grid, ov)
    fs, rect, pr, prc = plan.layout()
    sh, placed = plan.periodic_layout()
    fo, ro, po = oracle.geometry(H, H, m, offs, grid[0], grid[1], ov, periodic=True, placed=True)
    pro, sho, prco = oracle.pairs(ro, H, H, periodic=True, shifts=True)
    assert np.array_equal(fs, fo) and np.array_equal(rect, ro) and np.array_equal(placed, po)
    assert np.array_equal(pr, pro) and np.array_equal(sh, sho) and np.array_equal(prc, prco)
    assert (sh != 0).any()  # pairs across the boundary exist
    plan.close()


@pytest.mark.parametrize("blind", [False, True])
@pytest.mark.parametrize("case", CASES, ids=[f"m{c[1]}_{c[4][0]}x{c[4][1]}" for c in CASES])
def test_periodic_one_iteration_matches_the_oracle(case, blind):
    """One iteration from a scrambled state: every multiplier and the pairs
    across the boundary (and a subdomain's pairs with itself, 1 x 1) are used."""
    H, m, step, jit, grid, ov = case
    offs, u, w, f = _torus_case(H, m, step, jit, seed=2 * H + m)
    plan, ref = _pair(H, m, offs, w, f, grid, ov, blind=blind)
    _scramble(plan, ref, 5, blind)
    od.od2p_iterate(plan, 1)
    ref.iterate(1)
    out = _compare(plan, ref, blind)
    rf, re = od.od2p_metrics(plan)
    rfo, reo = ref.metrics()
    assert abs(rf - rfo) <= 1e-5 * rfo and abs(re - reo) <= 1e-4 * reo
    record(f"periodic_{'blind_' if blind else ''}m{m}_{grid[0]}x{grid[1]}_one_iteration", **out)
    plan.close()


@pytest.mark.parametrize("m64_kind", [0, 2])
def test_periodic_run_merge_snr_and_consensus(m64_kind):
    """30 iterations from u = 1 (m = 64, both transform splits): the state, the
    merged image (every copy of a pixel averaged), the SNR against the truth and
    the consensus residual follow the oracle."""
    H, m, step, jit, grid, ov = 192, 64, 16, 2, (2, 3), 16
    offs, u, w, f = _torus_case(H, m, step, jit, seed=11)
    plan, ref = _pair(H, m, offs, w, f, grid, ov, eta=0.5, r=0.3)
    od.ptycho_plan_set_fft(plan, m64_kind)
    od.od2p_iterate(plan, 30)
    ref.iterate(30)
    out = _compare(plan, ref, False, tol=1e-4)
    merged = od.od2p_merge(plan).cpu().numpy()
    out["merge"] = rel_l2(merged, ref.merge())
    assert out["merge"] < 1e-4
    # the SNR of the merged image (every copy averaged) against the truth, as the oracle computes it
    snr = od.od2p_snr(plan, torch.from_numpy(u.astype(np.complex64)).to(DEV))
    assert abs(snr - oracle.snr(merged, u)) < 1e-3
    out["consensus"] = abs(od.od2p_consensus_residual(plan) - ref.consensus()) / ref.consensus()
    assert out["consensus"] < 1e-3
    record(f"periodic_m64_kind{m64_kind}_30_iterations", **out)
    plan.close()


def test_periodic_step0_reads_u0_modulo_the_image():
    """Extended-coordinate rectangles start from u0 at (R mod H, C mod W), bit for bit."""
    H, m, step, jit, grid, ov = 128, 32, 8, 2, (2, 2), 8
    offs, u, w, f = _torus_case(H, m, step, jit, seed=12)
    u0 = u.astype(np.complex64)
    plan, ref = _pair(H, m, offs, w, f, grid, ov, u0=u0)
    assert np.array_equal(od.od2p_get_state(plan, od.STATE_U).cpu().numpy(), ref.get(oracle.U).astype(np.complex64))
    # the merge of a consistent state is the image itself (the average of equal copies)
    np.testing.assert_allclose(od.od2p_merge(plan).cpu().numpy(), u0, rtol=1e-6, atol=1e-7)
    plan.close()


def test_periodic_equals_vacuum_when_nothing_wraps():
    """Overlap 0 and a scan inside the image: no rectangle reaches across the
    boundary, so the periodic plan iterates exactly as the vacuum one."""
    H, m, step = 128, 32, 8
    offs = np.array([(r, c) for r in range(0, H - m + 1, step) for c in range(0, H - m + 1, step)], np.int32)
    rng = np.random.default_rng(13)
    w = ((0.5 + rng.random((m, m))) * np.exp(1j * rng.uniform(-2, 2, (m, m)))).astype(np.complex64)
    f = torch.from_numpy(rng.random((len(offs), m, m)).astype(np.float32)).to(DEV)
    plans = []
    for per in (False, True):
        g = od.Geometry(H, H, m, offs, 2, 2, 0, 0.5, 0.3, 0.2, periodic=per)
        p = od.ptycho_plan(g, f)
        od.od2p_init(p, torch.from_numpy(w).to(DEV))
        od.od2p_iterate(p, 3)
        plans.append(p)
    for k in (od.STATE_U, od.STATE_GAMMA, od.STATE_LAMBDA):
        assert torch.equal(od.od2p_get_state(plans[0], k), od.od2p_get_state(plans[1], k)), k
    for p in plans:
        p.close()


def test_periodic_is_deterministic():
    H, m, step, jit, grid, ov = 96, 16, 6, 1, (3, 3), 8
    offs, u, w, f = _torus_case(H, m, step, jit, seed=14)
    states = []
    for _ in range(2):
        plan, _ref = _pair(H, m, offs, w, f, grid, ov, blind=True)
        od.od2p_iterate(plan, 4)
        states.append([od.od2p_get_state(plan, k).clone() for k in (od.STATE_U, od.STATE_LAMBDA, od.STATE_W)])
        plan.close()
    for a, b in zip(*states):
        assert torch.equal(a, b)


@pytest.mark.parametrize("m", [32, 64, 256])
def test_periodic_image_space_operators_match_the_oracle(m):
    """Forward operator, overlap-add (adjoint) and the ST-AGM loss with both
    gradients on a periodic plan, windows wrapping around the image, against the
    oracle's periodic operators; the gradient frames stored and reused give the
    same gradients bit for bit."""
    H, step = (4 * m, m // 2) if m < 256 else (512, 64)
    offs, u, w, f = _torus_case(H, m, step, 2, seed=m + 3)
    g = od.Geometry(H, H, m, offs, 2, 2, 8, 0.5, 0.3, 0.2, periodic=True)
    plan = od.ptycho_plan(g, torch.from_numpy(np.asarray(f, np.float32)).to(DEV))
    u32, w32 = u.astype(np.complex64), w.astype(np.complex64)
    ud, wd = torch.from_numpy(u32).to(DEV), torch.from_numpy(w32).to(DEV)
    out = {}
    fr = od.ptycho_forward(plan, ud, wd).cpu().numpy()
    out["forward"] = rel_l2(fr, oracle.forward(u32, w32, offs, periodic=True))
    assert out["forward"] < TOL
    rng = np.random.default_rng(m)
    y = (rng.standard_normal(fr.shape) + 1j * rng.standard_normal(fr.shape)).astype(np.complex64)
    img = od.overlap_add(plan, torch.from_numpy(y).to(DEV), wd, ifft=True).cpu().numpy()
    out["adjoint"] = rel_l2(img, oracle.adjoint(y, w32, offs, H, H, periodic=True))
    assert out["adjoint"] < TOL
    loss, gu, gw = od.stagm_loss_grad(plan, ud, wd)
    lo, guo, gwo = oracle.loss_grad(u32, w32, offs, np.asarray(f, np.float32), 0.5, periodic=True)
    out["loss"] = abs(float(loss.item()) - lo) / lo
    out["grad_u"] = rel_l2(gu.cpu().numpy(), guo)
    out["grad_w"] = rel_l2(gw.cpu().numpy(), gwo)
    assert out["loss"] < TOL and out["grad_u"] < TOL and out["grad_w"] < TOL, out
    loss_s, _, _ = od.stagm_loss_grad(plan, ud, wd, grad_u=False, grad_w=False, recompute=od.STORE)
    _, gu2, gw2 = od.stagm_loss_grad(plan, ud, wd, recompute=od.FROM_STORE)
    assert torch.equal(gu2, gu) and torch.equal(gw2, gw) and float(loss_s.item()) == float(loss.item())
    record(f"periodic_image_operators_m{m}", **out)
    plan.close()
