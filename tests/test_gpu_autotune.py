"""Launch shapes of the frame update and the autotuner that picks one.

Every (variant, blocks-per-SM cap) must give the same iterates bit for bit --
the shape only changes which thread runs which butterfly, never the arithmetic
-- and tuning must leave the plan's state as it found it.
"""
import json

import numpy as np
import pytest
import torch

import paper_2011_00162_gb300 as od
from paper_2011_00162_gb300 import autotune, synth
from paper_2011_00162_gb300 import build as odbuild

from _cases import make_case

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    odbuild.build()


def _plan(p, blind=False):
    offs, u_true, w, f = make_case(p)
    g = od.Geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px, p.eps, p.eta, p.r,
                    mu=2.0 if blind else 0.0, gamma=0.1 if blind else 0.0, blind=blind)
    plan = od.ptycho_plan(g, torch.from_numpy(np.asarray(f, np.float32)).to(DEV))
    w0 = torch.from_numpy(np.asarray(w, np.complex64)).to(DEV)
    if blind:
        w0 = w0 * (1 + 0.05 * torch.randn(w0.shape, generator=torch.Generator().manual_seed(4)).to(DEV))
    od.od2p_init(plan, w0)
    return plan


def _states(plan, blind):
    sel = [od.STATE_U, od.STATE_GAMMA, od.STATE_LAMBDA] + (
        [od.STATE_WD, od.STATE_DELTA, od.STATE_W] if blind else [])
    return {k: od.od2p_get_state(plan, k).clone() for k in sel}


CASES = [(16, (5, 4), 120, 6, False), (32, (2, 3), 200, 10, False), (64, (2, 2), 256, 16, False),
         (128, (2, 2), 384, 32, False), (32, (2, 2), 160, 8, True), (64, (1, 2), 192, 16, True),
         (48, (2, 2), 192, 12, False), (80, (2, 2), 240, 20, False), (96, (2, 2), 288, 24, True),
         (256, (2, 2), 512, 64, False), (256, (2, 3), 560, 48, True)]


@pytest.mark.parametrize("m,grid,n,step,blind", CASES)
def test_every_launch_shape_gives_identical_iterates(m, grid, n, step, blind):
    p = synth.Problem("t", n, m, step, 2, grid[0], grid[1], 12, 1e5, 1, eta=0.3, r=0.2, seed=m)
    ref = _plan(p, blind)
    od.od2p_iterate(ref, 3)
    want = _states(ref, blind)
    rf_ref, re_ref = od.od2p_metrics(ref)
    assert od.ptycho_plan_get_launch(ref)[:2] == (0, 0)
    for v in range(od.LAUNCH_VARIANTS):
        od.ptycho_plan_set_launch(ref, v, 0)
        most = od.ptycho_plan_get_launch(ref)[2]
        assert most >= 1
        for cap in sorted({1, most}):
            plan = _plan(p, blind)
            od.ptycho_plan_set_launch(plan, v, cap)
            # m = 256 has no block cap (reported as 0)
            assert od.ptycho_plan_get_launch(plan) == (v, cap if m != 256 else 0, most)
            od.od2p_iterate(plan, 3)
            got = _states(plan, blind)
            rf, re = od.od2p_metrics(plan)
            if m == 256 and v != 0:
                # m = 256: the cluster variant is a different kernel sequence, whose
                # FP32 contractions the compiler may choose differently: equal to
                # rounding (both are compared with the FP64 oracle in the parity tests)
                for k in want:
                    d = float(torch.linalg.vector_norm(got[k] - want[k]) /
                              max(float(torch.linalg.vector_norm(want[k])), 1e-30))
                    assert d <= 1e-5, (v, k, d)
                assert abs(rf - rf_ref) <= 1e-5 * abs(rf_ref) and abs(re - re_ref) <= 1e-3 * abs(re_ref)
                plan.close()
                continue
            for k in want:
                assert torch.equal(got[k], want[k]), (v, cap, k)
            # RF partials are grouped per warp of a frame group: same value up to summation order
            assert abs(rf - rf_ref) <= 1e-5 * abs(rf_ref) and re == re_ref
            plan.close()
    ref.close()


def test_switching_shape_mid_run_keeps_iterates():
    p = synth.Problem("t", 256, 64, 16, 2, 2, 2, 12, 1e5, 1, eta=0.3, r=0.2, seed=5)
    a, b = _plan(p), _plan(p)
    od.od2p_iterate(a, 4)
    od.od2p_iterate(b, 1)
    od.ptycho_plan_set_launch(b, 1, 1)
    od.od2p_iterate(b, 2)
    od.ptycho_plan_set_launch(b, 0, 0)
    od.od2p_iterate(b, 1)
    for k, t in _states(a, False).items():
        assert torch.equal(t, _states(b, False)[k])


def test_set_launch_argument_errors():
    p = synth.Problem("t", 120, 16, 6, 2, 2, 2, 12, 1e5, 1, seed=2)
    plan = _plan(p)
    for v, b in [(-1, 0), (od.LAUNCH_VARIANTS, 0), (0, -1)]:
        with pytest.raises(od.PtychoError) as e:
            od.ptycho_plan_set_launch(plan, v, b)
        assert e.value.code == 1  # PTYCHO_ERR_INVALID_ARG
    # a cap above what fits is clamped, not refused
    od.ptycho_plan_set_launch(plan, 0, 1000)
    assert od.ptycho_plan_get_launch(plan)[1] == 1000
    # m = 256: variant 0 is the three passes, 1 the cluster launch; no block cap
    p256 = synth.Problem("t", 512, 256, 64, 2, 2, 2, 12, 1e5, 1, seed=3)
    plan256 = _plan(p256)
    od.ptycho_plan_set_launch(plan256, 0, 3)
    assert od.ptycho_plan_get_launch(plan256) == (0, 0, 1)
    # the three passes run in waves dealt to chains (at most one chain per wave)
    wf, ch, ln = od.ptycho_plan_get_waves(plan256)
    n_waves = -(-plan256.n_frames // wf)
    assert wf > 0 and 1 <= ch <= n_waves and ln == 3 * n_waves
    od.ptycho_plan_set_launch(plan256, 1, 0)
    assert od.ptycho_plan_get_launch(plan256) == (1, 0, 1)
    assert od.ptycho_plan_get_waves(plan256) == (0, 1, 1)
    assert od.ptycho_plan_get_waves(plan) == (0, 1, 1)


def test_tune_plan_restores_state_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    p = synth.Problem("t", 256, 32, 10, 2, 2, 2, 12, 1e5, 1, eta=0.3, r=0.2, seed=8)
    plan = _plan(p)
    od.od2p_iterate(plan, 2)
    before = _states(plan, False)
    entry = autotune.tune_plan(plan, n_iter=3, warmup=1, path=path)
    assert entry["cached"] is False
    assert (entry["variant"], entry["blocks_per_sm"]) == od.ptycho_plan_get_launch(plan)[:2]
    assert entry["us"] == min(entry["trials"].values())
    for k, t in _states(plan, False).items():
        assert torch.equal(t, before[k]), k
    # the tuned plan continues exactly like an untuned one
    ref = _plan(p)
    od.od2p_iterate(ref, 2)
    od.od2p_iterate(plan, 2)
    od.od2p_iterate(ref, 2)
    for k, t in _states(plan, False).items():
        assert torch.equal(t, _states(ref, False)[k]), k
    doc = json.load(open(path))
    assert len(doc["entries"]) == 1
    # a second plan of the same workload takes the cached shape without timing
    again = _plan(p)
    od.ptycho_plan_set_launch(again, 1 - entry["variant"], 0)
    hit = autotune.tune_plan(again, path=path)
    assert hit["cached"] is True
    assert od.ptycho_plan_get_launch(again)[:2] == (entry["variant"], entry["blocks_per_sm"])


def test_batch_launch_shapes_and_tuning(tmp_path):
    probs = [p for p in synth.batched_problems(40, seed=3) if p.n <= 400][:5]
    cases = [make_case(p, noise_seed=i) for i, p in enumerate(probs)]
    geoms = [od.Geometry(p.n, p.n, p.m, c[0], p.sub_rows, p.sub_cols, p.overlap_px, 0.5, 2.0, 0.5)
             for p, c in zip(probs, cases)]
    fs = [torch.from_numpy(np.asarray(c[3], np.float32)).to(DEV) for c in cases]

    def run(variant, cap, tune=False):
        batch = od.ptycho_batch_plan(geoms, fs)
        for mb, c in zip(batch.members, cases):
            od.od2p_init(mb, torch.from_numpy(np.asarray(c[2], np.complex64)).to(DEV))
        if tune:
            entry = autotune.tune_batch(batch, n_iter=3, warmup=1, path=str(tmp_path / "b.json"))
            assert entry["cached"] is False
        else:
            od.ptycho_batch_set_launch(batch, variant, cap)
            assert od.ptycho_batch_get_launch(batch) == (variant, cap)
        batch.iterate(3)
        out = [_states(mb, False) for mb in batch.members]
        # a member's launch shape belongs to the batch
        with pytest.raises(od.PtychoError) as e:
            od.ptycho_plan_set_launch(batch.members[0], 0, 0)
        assert e.value.code == 6  # PTYCHO_ERR_STATE
        batch.close()
        return out

    ref = run(0, 0)
    for variant, cap, tune in [(1, 0, False), (1, 1, False), (0, 1, False), (0, 0, True)]:
        got = run(variant, cap, tune)
        for a, b in zip(got, ref):
            for k in a:
                assert torch.equal(a[k], b[k]), (variant, cap, tune, k)


def test_tune_plan_times_the_transform_kinds_for_m64(tmp_path):
    """For m = 64 the tuner also times the 16 x 4 transform kinds, applies the
    fastest candidate and restores the state; fft=False keeps to shapes."""
    path = str(tmp_path / "tune.json")
    p = synth.Problem("t64", 256, 64, 16, 2, 2, 2, 16, 1e4, 1, eta=2.0, r=0.5, seed=8)
    plan = _plan(p)
    od.od2p_iterate(plan, 2)
    before = _states(plan, False)
    entry = autotune.tune_plan(plan, n_iter=3, warmup=1, path=path)
    assert {"fft1", "fft2"} <= set(entry["trials"]) and entry["fft"] in (0, 1, 2)
    assert od.ptycho_plan_get_fft(plan) == entry["fft"]
    assert entry["us"] == min(entry["trials"].values())
    for k, t in _states(plan, False).items():
        assert torch.equal(t, before[k]), k
    again = _plan(p)
    hit = autotune.tune_plan(again, path=path)
    assert hit["cached"] is True and od.ptycho_plan_get_fft(again) == entry["fft"]
    shapes_only = autotune.tune_plan(_plan(p), n_iter=2, warmup=1, path=path, fft=False)
    assert not any(k.startswith("fft") for k in shapes_only["trials"]) and shapes_only["fft"] == 0


@pytest.mark.parametrize("blind", [False, True])
def test_m256_wave_shapes_give_identical_iterates(tmp_path, blind):
    """m = 256: every wave shape (frames per wave, chains side by side) gives the
    same iterates bit for bit, reports its launches, and the tuner picks one of
    its shapes and caches it."""
    p = synth.Problem("w", 512, 256, 32, 2, 2, 2, 12, 1e5, 1, eta=2.0, r=0.5, seed=6)
    ref = _plan(p, blind)
    J = ref.n_frames
    od.od2p_iterate(ref, 2)
    want = _states(ref, blind)
    for wf, ch in [(1, 1), (5, 3), (19, 4), (40, 8), (152, 2)]:
        pl = _plan(p, blind)
        od.ptycho_plan_set_waves(pl, wf, ch)
        n_waves = -(-J // wf)
        assert od.ptycho_plan_get_waves(pl) == (wf, min(ch, n_waves), 3 * n_waves)
        od.od2p_iterate(pl, 2)
        for k, t in _states(pl, blind).items():
            assert torch.equal(t, want[k]), (wf, ch, k)
        pl.close()
    for bad in [(0, 1), (153, 1), (4, 0), (4, 9)]:
        with pytest.raises(od.PtychoError) as e:
            od.ptycho_plan_set_waves(ref, *bad)
        assert e.value.code == 1  # PTYCHO_ERR_INVALID_ARG
    small = _plan(synth.Problem("s", 64, 16, 8, 0, 1, 1, 0, None, 1))
    with pytest.raises(od.PtychoError):
        od.ptycho_plan_set_waves(small, 4, 2)
    # the tuner times its wave shapes for the three passes and caches the choice
    od.ptycho_plan_set_launch(ref, 0, 0)
    entry = autotune.tune_plan(ref, n_iter=2, warmup=1, path=str(tmp_path / "w.json"))
    if entry["variant"] == 0:
        assert tuple(entry["waves"]) in autotune.WAVE_SHAPES
        assert od.ptycho_plan_get_waves(ref)[:2] == (entry["waves"][0], min(entry["waves"][1], -(-J // entry["waves"][0])))
        again = _plan(p, blind)
        assert autotune.tune_plan(again, path=str(tmp_path / "w.json"))["cached"] is True
        assert od.ptycho_plan_get_waves(again)[:2] == od.ptycho_plan_get_waves(ref)[:2]
