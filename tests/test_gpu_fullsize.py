"""Full-size blind parity (Algorithm 3, section 3.2) against the FP64 oracle.

The two blind workloads at their full sizes, through the C ABI:

* 4096^2 image, 6561 frames of 256^2, 8x8 subdomains, Poisson 1e5: a short run
  from Step 0 (merged image and probe after global-phase alignment), then one
  whole iteration from a scrambled state with every state array compared --
  the frame update, the probe update over D = 64 subdomains and the 8x8 list
  gather of the U-update -- for both launch variants of the frame update;
* 1024^2 image, 841 frames of 128^2, 4x4 subdomains, Poisson 1e4: a 100-
  iteration run from Step 0, the merged image and the probe compared after
  global-phase alignment.

Tolerances are the build's: one iteration within 1e-5 relative L2 per state
array, a run within 1e-3 after global-phase alignment.  The oracle holds about
35 GB of FP64 state for the large workload on the host.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2011_00162_gb300 as od
from paper_2011_00162_gb300 import synth
from paper_2011_00162_gb300 import build as odbuild

from _cases import record

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
ONE_ITER_TOL = 1e-5
END_TOL = 1e-3
BLIND = dict(eta=2.0, r=0.5, mu=1.0, gamma=0.1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    odbuild.build()


def _rel_l2(a, b, chunk=1 << 24) -> float:
    """||a - b|| / ||b|| over flat arrays, in chunks (the arrays hold ~4e8 values)."""
    a, b = np.asarray(a).reshape(-1), np.asarray(b).reshape(-1)
    num = den = 0.0
    for k in range(0, b.size, chunk):
        bb = b[k:k + chunk].astype(np.complex128)
        num += float(np.sum(np.abs(a[k:k + chunk].astype(np.complex128) - bb) ** 2))
        den += float(np.sum(np.abs(bb) ** 2))
    return float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num))


def _phase_aligned(x, ref) -> float:
    x = np.asarray(x, np.complex128).reshape(-1)
    ref = np.asarray(ref, np.complex128).reshape(-1)
    th = np.angle(np.vdot(x, ref))
    return float(np.linalg.norm(x * np.exp(1j * th) - ref) / np.linalg.norm(ref))


def _intensities(p, seed):
    offs = p.offsets()
    u_true, w_true = p.truth(), p.probe()
    f = np.empty((len(offs), p.m, p.m), np.float32)
    clean = np.empty((len(offs), p.m, p.m), np.float64)
    for j0 in range(0, len(offs), 256):  # the oracle's forward operator in slices (memory)
        clean[j0:j0 + 256] = np.abs(oracle.forward(u_true, w_true, offs[j0:j0 + 256])) ** 2
    f[:] = synth.poissonize(clean, p.peak, seed)
    del clean
    return offs, f


def _pair(p, offs, f, w0):
    g = od.Geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px, eps=p.eps, blind=True, **BLIND)
    plan = od.ptycho_plan(g, torch.from_numpy(f).to(DEV))
    od.od2p_init(plan, torch.from_numpy(w0.astype(np.complex64)).to(DEV))
    ref = oracle.ADMM(f, w0, offs, p.n, p.n, p.sub_rows, p.sub_cols, p.overlap_px, p.eps, BLIND["eta"], BLIND["r"],
                      blind=True, mu=BLIND["mu"], gamma=BLIND["gamma"])
    return plan, ref


def _end_of_run(plan, ref, p):
    u = od.od2p_merge(plan).cpu().numpy()
    w = od.od2p_get_state(plan, od.STATE_W).cpu().numpy()
    return _phase_aligned(u, ref.merge()), _phase_aligned(w, ref.get(oracle.W))


SEL = [("u", od.STATE_U, oracle.U), ("Gamma", od.STATE_GAMMA, oracle.GAMMA), ("Lambda", od.STATE_LAMBDA, oracle.LAMBDA),
       ("W_d", od.STATE_WD, oracle.WD), ("Delta", od.STATE_DELTA, oracle.DELTA), ("w", od.STATE_W, oracle.W)]


def test_large_blind_full_size_run_and_whole_iteration():
    p = synth.large_blind()
    offs, f = _intensities(p, 11)
    assert len(offs) == 6561 and p.sub_rows * p.sub_cols == 64
    w0 = synth.gaussian_probe(p.m)
    plan, ref = _pair(p, offs, f, w0)
    # ---- a short run from Step 0: merged image and probe after phase alignment
    n_it = 5
    od.od2p_iterate(plan, n_it)
    ref.iterate(n_it)
    eu, ew = _end_of_run(plan, ref, p)
    record("config5_end_of_run_5_iterations", u=eu, w=ew)
    assert eu < END_TOL and ew < END_TOL, (eu, ew)
    # ---- one whole iteration from a scrambled state, every state array
    rng = np.random.default_rng(12)
    start = {}
    for name, wg, wo in SEL[:5]:
        cur = ref.get(wo)
        n = cur.size
        if name in ("u", "W_d"):
            v = cur * (1 + 0.1 * (rng.standard_normal(n) + 1j * rng.standard_normal(n)))
        else:
            scale = 0.2 * (np.abs(cur).mean() + 1e-3) if name == "Gamma" else 0.2
            v = scale * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
        start[name] = v.astype(np.complex64)
        del cur, v
        ref.set(wo, start[name])
    ref.iterate(1)
    want = {name: ref.get(wo) for name, _, wo in SEL}
    for variant in (0, 1):  # three passes over an L2 intermediate; one cluster launch
        od.ptycho_plan_set_launch(plan, variant, 0)
        for name, wg, _ in SEL[:5]:
            od.od2p_set_state(plan, wg, torch.from_numpy(start[name]).to(DEV))
        od.od2p_iterate(plan, 1)
        errs = {}
        for name, wg, _ in SEL:
            errs[name] = _rel_l2(od.od2p_get_state(plan, wg).cpu().numpy(), want[name])
        record(f"config5_one_iteration_scrambled_variant{variant}", **errs)
        for name, e in errs.items():
            assert e < ONE_ITER_TOL, (variant, name, e)
    plan.close()


def test_blind_1024_full_run_100_iterations():
    p = synth.blind_4x4()
    offs, f = _intensities(p, 7)
    assert len(offs) == 841
    w0 = synth.gaussian_probe(p.m)
    plan, ref = _pair(p, offs, f, w0)
    od.od2p_iterate(plan, 100)
    ref.iterate(100)
    eu, ew = _end_of_run(plan, ref, p)
    rf_g, re_g = od.od2p_metrics(plan)
    rf_o, re_o = ref.metrics()
    record("config4_end_of_run_100_iterations", u=eu, w=ew, rf=abs(rf_g - rf_o) / rf_o)
    assert eu < END_TOL and ew < END_TOL, (eu, ew)
    assert abs(rf_g - rf_o) < END_TOL * rf_o
    plan.close()
