"""Penalty changes between iterations, the consensus residual and the
residual-balancing driver, against the FP64 oracle doing the same."""
import numpy as np
import pytest
import torch

import oracle
import paper_2011_00162_gb300 as od
from paper_2011_00162_gb300 import adaptive, synth
from paper_2011_00162_gb300 import build as odbuild

from _cases import make_case, record, rel_l2

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    odbuild.build()


def _pair(p, eta, r, blind=False):
    offs, u_true, w, f = make_case(p)
    g = od.Geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px, p.eps, eta, r,
                    mu=1.0 if blind else 0.0, blind=blind)
    plan = od.ptycho_plan(g, torch.from_numpy(np.asarray(f, np.float32)).to(DEV))
    od.od2p_init(plan, torch.from_numpy(np.asarray(w, np.complex64)).to(DEV))
    ref = oracle.ADMM(f, w, offs, p.n, p.n, p.sub_rows, p.sub_cols, p.overlap_px, p.eps, eta, r, blind=blind,
                      mu=1.0 if blind else 0.0)
    return plan, ref


def _states_close(plan, ref, tol, blind=False):
    sel = [(od.STATE_U, oracle.U), (od.STATE_GAMMA, oracle.GAMMA), (od.STATE_LAMBDA, oracle.LAMBDA)]
    if blind:
        sel += [(od.STATE_WD, oracle.WD), (od.STATE_W, oracle.W)]
    out = {}
    for k, ko in sel:
        b = ref.get(ko)
        if b.size:
            out[str(k)] = rel_l2(od.od2p_get_state(plan, k).cpu().numpy(), b)
    assert all(v < tol for v in out.values()), out
    return out


@pytest.mark.parametrize("m,blind", [(64, False), (32, True), (256, False)])
def test_penalty_change_matches_oracle(m, blind):
    n = {64: 256, 32: 128, 256: 512}[m]
    p = synth.Problem("pen", n, m, m // 4, 2, 2, 2, 16, 1e4, 1, seed=m)
    plan, ref = _pair(p, 2.0, 0.5, blind)
    ref.iterate(2)
    # start both from the oracle's state, so that each comparison measures the
    # penalty change and one iteration only
    sel = [(od.STATE_U, oracle.U), (od.STATE_GAMMA, oracle.GAMMA), (od.STATE_LAMBDA, oracle.LAMBDA)]
    if blind:
        sel += [(od.STATE_WD, oracle.WD), (od.STATE_DELTA, oracle.DELTA), (od.STATE_W, oracle.W)]
    for k, ko in sel:
        v = ref.get(ko)
        if v.size:
            od.od2p_set_state(plan, k, torch.from_numpy(v.astype(np.complex64)).to(DEV))
    for eta, r in [(3.0, 1.5), (1.5, 0.25)]:
        od.od2p_set_penalties(plan, eta, r)
        ref.set_penalties(eta, r)
        out = _states_close(plan, ref, TOL, blind)   # the rescaled multipliers
        od.od2p_iterate(plan, 1)
        ref.iterate(1)
        out = _states_close(plan, ref, TOL, blind)   # one iteration at the new penalties
    record(f"penalty_change_m{m}_{'blind' if blind else 'nonblind'}", **out)
    rc = od.od2p_consensus_residual(plan)
    assert abs(rc - ref.consensus()) <= 1e-5 * max(ref.consensus(), 1e-30) + 1e-7


def test_balanced_run_replays_on_the_oracle():
    """The driver's schedule of r, replayed on the oracle, gives the same iterates."""
    p = synth.Problem("bal", 256, 64, 16, 2, 2, 2, 16, 1e4, 1, seed=9)
    plan, ref = _pair(p, 2.0, 0.02)  # a small r: the copies drift apart, r goes up
    hist = adaptive.iterate_balanced(plan, 40, every=10)
    rs = [h["r"] for h in hist]
    assert rs[0] > 0.02 or len(set(rs)) > 1, hist
    r_prev = 0.02
    for h in hist:
        ref.iterate(10)
        if h["r"] != r_prev:
            ref.set_penalties(2.0, h["r"])
            r_prev = h["r"]
    u, uo = od.od2p_get_state(plan, od.STATE_U).cpu().numpy(), ref.get(oracle.U)
    err = rel_l2(u, uo)
    record("balanced_run_40its", u=err, r_final=rs[-1])
    assert err < 1e-4, (err, hist)
    assert abs(hist[-1]["consensus"] - ref.consensus()) < 1e-3 * ref.consensus() + 1e-7


def test_penalty_arguments_and_batch_members():
    p = synth.Problem("pa", 64, 16, 4, 0, 1, 2, 8, None, 1, seed=1)
    plan, _ = _pair(p, 0.1, 0.05)
    for eta, r in [(0.0, 1.0), (-1.0, 1.0), (1.0, -1.0), (float("nan"), 1.0)]:
        with pytest.raises(od.PtychoError):
            od.od2p_set_penalties(plan, eta, r)
    one = od.ptycho_plan(od.Geometry(64, 64, 16, p.offsets()), torch.ones((169, 16, 16), device=DEV))
    assert od.od2p_consensus_residual(one) == 0.0 or one.n_pairs > 0
    offs, u_true, w, f = make_case(p)
    g = od.Geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px, 0.5, 0.1, 0.05)
    batch = od.ptycho_batch_plan([g], [torch.from_numpy(np.asarray(f, np.float32)).to(DEV)])
    with pytest.raises(od.PtychoError) as e:
        od.od2p_set_penalties(batch.members[0], 1.0, 1.0)
    assert e.value.code == 6
    batch.close()


@pytest.mark.parametrize("which", ["small_2sub", "grid_4x4"])
def test_operator_norms_match_oracle(which):
    """Lemma 2.4's operator norms from the plan's illumination equal the oracle's,
    and the selected (r, eta) lie in K; blind plans are refused."""
    p = getattr(synth, which)()
    offs, u_true, w, f = make_case(p)
    g = od.Geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px, p.eps, p.eta, p.r)
    plan = od.ptycho_plan(g, torch.as_tensor(np.asarray(f, np.float32), device=DEV))
    od.od2p_init(plan, torch.as_tensor(np.asarray(w, np.complex64), device=DEV))
    a, b = od.od2p_operator_norms(plan)
    a_want, b_want = oracle.operator_norms(w, offs, p.n, p.n, p.sub_rows, p.sub_cols, p.overlap_px)
    record(f"operator_norms_{which}", gpu=[a, b], oracle=[a_want, b_want])
    assert abs(a - a_want) <= 1e-6 * a_want and abs(b - b_want) <= 1e-6 * b_want, (a, a_want, b, b_want)
    r, eta = adaptive.select_in_K(plan)
    assert adaptive.in_K(r, eta, (a_want, b_want), p.eps)
    gb = od.Geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px, p.eps, 2.0, 0.5,
                     mu=1.0, gamma=0.1, blind=True)
    bp = od.ptycho_plan(gb, torch.as_tensor(np.asarray(f, np.float32), device=DEV))
    od.od2p_init(bp, torch.as_tensor(np.asarray(w, np.complex64), device=DEV))
    with pytest.raises(RuntimeError):
        od.od2p_operator_norms(bp)


def test_frame_residual_matches_oracle():
    """||Gamma^{n+1} - Gamma^n|| / ||sqrt f|| across one iteration equals the
    oracle's, and a snapshot is required first."""
    p = synth.Problem("fres", 192, 32, 8, 1, 2, 2, 8, 1e4, 1, seed=5)
    plan, ref = _pair(p, 2.0, 0.5)
    with pytest.raises(RuntimeError):
        od.od2p_frame_residual(plan)
    od.od2p_iterate(plan, 2)
    ref.iterate(2)
    od.od2p_gamma_snapshot(plan)
    g0 = ref.get(oracle.GAMMA)
    od.od2p_iterate(plan, 1)
    ref.iterate(1)
    got = od.od2p_frame_residual(plan)
    offs, _, _, f = make_case(p)
    want = np.linalg.norm(ref.get(oracle.GAMMA) - g0) / np.sqrt(np.sum(np.asarray(f, np.float64)))
    record("frame_residual", gpu=got, oracle=want)
    assert abs(got - want) < 1e-4 * want, (got, want)


def test_balanced_eta_run_replays_on_the_oracle():
    """The driver's schedule of (eta, r), replayed on the oracle, gives the same iterates."""
    p = synth.Problem("bal2", 256, 64, 16, 2, 2, 2, 16, 1e4, 1, seed=9)
    plan, ref = _pair(p, 8.0, 0.02)
    hist = adaptive.iterate_balanced(plan, 40, every=10, balance_eta=True)
    assert len({(h["eta"], h["r"]) for h in hist}) > 1, hist
    eta_prev, r_prev = 8.0, 0.02
    for h in hist:
        ref.iterate(10)
        if (h["eta"], h["r"]) != (eta_prev, r_prev):
            ref.set_penalties(h["eta"], h["r"])
            eta_prev, r_prev = h["eta"], h["r"]
    err = rel_l2(od.od2p_get_state(plan, od.STATE_U).cpu().numpy(), ref.get(oracle.U))
    record("balanced_eta_run_40its", u=err, eta_final=hist[-1]["eta"], r_final=hist[-1]["r"])
    # a 40-iteration noisy run with penalty jumps: the end-of-run bar (1e-3), not the one-iteration one
    assert err < 1e-3, (err, hist)
    assert all(h["eta"] > (1 - p.eps) / p.eps for h in hist)
