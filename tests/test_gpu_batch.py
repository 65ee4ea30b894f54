"""Batched reconstructions: one persistent frame-update launch per probe side and
one subdomain-update launch per iteration, against each member run alone."""
import numpy as np
import pytest
import torch

import oracle
import paper_2011_00162_gb300 as od
from paper_2011_00162_gb300 import build as odbuild
from paper_2011_00162_gb300 import synth

from _cases import make_case, record, rel_l2

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    odbuild.build()


def _members(count=6, seed=3, max_n=400):
    probs = [p for p in synth.batched_problems(40, seed=seed) if p.n <= max_n][:count]
    assert len({p.m for p in probs}) >= 2  # mixed probe sides in one batch
    cases = [make_case(p, noise_seed=i) for i, p in enumerate(probs)]
    geoms = [od.Geometry(p.n, p.n, p.m, c[0], p.sub_rows, p.sub_cols, p.overlap_px, 0.5, 2.0, 0.5)
             for p, c in zip(probs, cases)]
    return probs, cases, geoms


def test_batch_equals_members_run_alone_bitwise():
    probs, cases, geoms = _members()
    fs = [torch.from_numpy(c[3]).to(DEV) for c in cases]
    batch = od.ptycho_batch_plan(geoms, fs)
    for m, c in zip(batch.members, cases):
        od.od2p_init(m, torch.from_numpy(c[2]).to(DEV))
    batch.iterate(3)
    for i, (g, c) in enumerate(zip(geoms, cases)):
        alone = od.ptycho_plan(g, fs[i])
        od.od2p_init(alone, torch.from_numpy(c[2]).to(DEV))
        if g.m == 64:  # the batch runs m = 64 members on the 16 x 4 split
            od.ptycho_plan_set_fft(alone, 2)
        od.od2p_iterate(alone, 3)
        for k in (od.STATE_U, od.STATE_GAMMA, od.STATE_LAMBDA):
            assert torch.equal(od.od2p_get_state(batch.members[i], k), od.od2p_get_state(alone, k)), (i, k)
        alone.close()
    # a member iterated on its own is refused by the batch afterwards
    od.od2p_iterate(batch.members[0], 1)
    with pytest.raises(od.PtychoError):
        batch.iterate(1)
    batch.close()


def test_batch_member_matches_oracle():
    probs, cases, geoms = _members(count=3)
    fs = [torch.from_numpy(c[3]).to(DEV) for c in cases]
    batch = od.ptycho_batch_plan(geoms, fs)
    for m, c in zip(batch.members, cases):
        od.od2p_init(m, torch.from_numpy(c[2]).to(DEV))
    batch.iterate(1)
    for i, (p, c) in enumerate(zip(probs, cases)):
        offs, u_true, w, f = c
        ref = oracle.ADMM(f, w, offs, p.n, p.n, p.sub_rows, p.sub_cols, p.overlap_px, 0.5, 2.0, 0.5)
        ref.iterate(1)
        errs = {}
        for k, ko in ((od.STATE_U, oracle.U), (od.STATE_GAMMA, oracle.GAMMA), (od.STATE_LAMBDA, oracle.LAMBDA)):
            b = ref.get(ko)
            if b.size:
                errs[str(k)] = rel_l2(od.od2p_get_state(batch.members[i], k).cpu().numpy(), b)
                assert errs[str(k)] < 1e-5
        record(f"config3_member{i}_one_iteration", **errs)
    batch.close()


def test_batch_with_blind_and_dense_members_bitwise():
    """Blind members (frame-list gather, probe update between the two launches),
    a nonblind member with more than 255 frames over a pixel (frame-list gather
    with the known probe) and slot-gather members in one batch: every member
    equals itself iterated alone, and a blind member matches the oracle."""
    specs = [(32, 96, 8, True, 2, 31), (64, 192, 16, True, 2, 32), (16, 64, 4, False, 2, 33),
             (128, 384, 32, True, 2, 34), (32, 64, 2, False, 1, 35), (48, 144, 12, False, 2, 36)]
    probs, cases, geoms, w0s = [], [], [], []
    for m, n, step, blind, grid, seed in specs:
        p = synth.Problem(f"bb{m}", n, m, step, 0 if step < 4 else 1, grid, grid, 8, 1e4, 1, eta=2.0, r=0.5,
                          blind=blind, mu=1.0 if blind else 0.0, gamma=0.1 if blind else 0.0, seed=seed)
        c = make_case(p, noise_seed=seed)
        probs.append(p)
        cases.append(c)
        geoms.append(od.Geometry(p.n, p.n, p.m, c[0], p.sub_rows, p.sub_cols, p.overlap_px, 0.5, 2.0, 0.5,
                                 mu=p.mu, gamma=p.gamma, blind=blind))
        w0s.append(synth.gaussian_probe(m) if blind else np.asarray(c[2], np.complex64))
    fs = [torch.from_numpy(np.asarray(c[3], np.float32)).to(DEV) for c in cases]
    batch = od.ptycho_batch_plan(geoms, fs)
    for mb, w0 in zip(batch.members, w0s):
        od.od2p_init(mb, torch.from_numpy(w0).to(DEV))
    batch.iterate(3)
    for i, g in enumerate(geoms):
        alone = od.ptycho_plan(g, fs[i])
        od.od2p_init(alone, torch.from_numpy(w0s[i]).to(DEV))
        if g.m == 64:  # the batch runs m = 64 members on the 16 x 4 split
            od.ptycho_plan_set_fft(alone, 2)
        od.od2p_iterate(alone, 3)
        sel = [od.STATE_U, od.STATE_GAMMA, od.STATE_LAMBDA] + (
            [od.STATE_WD, od.STATE_DELTA, od.STATE_W] if g.blind else [])
        for k in sel:
            assert torch.equal(od.od2p_get_state(batch.members[i], k), od.od2p_get_state(alone, k)), (i, k)
        alone.close()
    # one blind member against the FP64 oracle (three iterations)
    i = 0
    p, (offs, u_true, w, f) = probs[i], cases[i]
    ref = oracle.ADMM(f, w0s[i], offs, p.n, p.n, p.sub_rows, p.sub_cols, p.overlap_px, 0.5, 2.0, 0.5, blind=True,
                      mu=p.mu, gamma=p.gamma)
    ref.iterate(3)
    for k, ko in ((od.STATE_U, oracle.U), (od.STATE_WD, oracle.WD), (od.STATE_W, oracle.W)):
        assert rel_l2(od.od2p_get_state(batch.members[i], k).cpu().numpy(), ref.get(ko)) < 1e-5, k
    batch.close()


def test_batch_with_mixed_radix_probe_sides_bitwise():
    """Probe sides 48, 80 and 96 (mixed-radix FFTs) beside 32 and 64 in one batch."""
    probs = [synth.Problem(f"b{m}", n, m, step, 1, 2, 2, 8, 1e4, 1, seed=m)
             for m, n, step in [(48, 192, 12), (80, 240, 20), (96, 288, 24), (32, 128, 8), (64, 256, 16), (48, 144, 12)]]
    cases = [make_case(p, noise_seed=i) for i, p in enumerate(probs)]
    geoms = [od.Geometry(p.n, p.n, p.m, c[0], p.sub_rows, p.sub_cols, p.overlap_px, 0.5, 2.0, 0.5)
             for p, c in zip(probs, cases)]
    fs = [torch.from_numpy(np.asarray(c[3], np.float32)).to(DEV) for c in cases]
    batch = od.ptycho_batch_plan(geoms, fs)
    for m, c in zip(batch.members, cases):
        od.od2p_init(m, torch.from_numpy(np.asarray(c[2], np.complex64)).to(DEV))
    batch.iterate(2)
    for i, (g, c) in enumerate(zip(geoms, cases)):
        alone = od.ptycho_plan(g, fs[i])
        od.od2p_init(alone, torch.from_numpy(np.asarray(c[2], np.complex64)).to(DEV))
        if g.m == 64:  # the batch runs m = 64 members on the 16 x 4 split
            od.ptycho_plan_set_fft(alone, 2)
        od.od2p_iterate(alone, 2)
        for k in (od.STATE_U, od.STATE_GAMMA, od.STATE_LAMBDA):
            assert torch.equal(od.od2p_get_state(batch.members[i], k), od.od2p_get_state(alone, k)), (i, k)
        alone.close()
    # one member against the oracle after one more iteration from the same state
    p, (offs, u_true, w, f) = probs[2], cases[2]
    ref = oracle.ADMM(f, w, offs, p.n, p.n, p.sub_rows, p.sub_cols, p.overlap_px, 0.5, 2.0, 0.5)
    for k, ko in ((od.STATE_U, oracle.U), (od.STATE_GAMMA, oracle.GAMMA), (od.STATE_LAMBDA, oracle.LAMBDA)):
        ref.set(ko, od.od2p_get_state(batch.members[2], k).cpu().numpy())
    batch.iterate(1)
    ref.iterate(1)
    for k, ko in ((od.STATE_U, oracle.U), (od.STATE_GAMMA, oracle.GAMMA), (od.STATE_LAMBDA, oracle.LAMBDA)):
        assert rel_l2(od.od2p_get_state(batch.members[2], k).cpu().numpy(), ref.get(ko)) < 1e-5
    batch.close()


def test_batch_with_m256_members_bitwise():
    """m = 256 members (blind and nonblind, several waves each) beside m = 32 and
    m = 64 members: each member equals itself iterated alone in the same launch
    variant, for the three wave passes and for the cluster launch; one m = 256
    member against the oracle."""
    specs = [(256, 512, 64, True, 2, 41), (32, 128, 8, False, 2, 42), (256, 448, 48, False, 2, 43),
             (64, 256, 16, True, 2, 44)]
    probs, cases, geoms, w0s = [], [], [], []
    for m, n, step, blind, grid, seed in specs:
        p = synth.Problem(f"b{m}", n, m, step, 1, grid, grid, 8, 1e4, 1, eta=2.0, r=0.5, blind=blind,
                          mu=1.0 if blind else 0.0, gamma=0.1 if blind else 0.0, seed=seed)
        c = make_case(p, noise_seed=seed)
        probs.append(p)
        cases.append(c)
        geoms.append(od.Geometry(p.n, p.n, p.m, c[0], p.sub_rows, p.sub_cols, p.overlap_px, 0.5, 2.0, 0.5,
                                 mu=p.mu, gamma=p.gamma, blind=blind))
        w0s.append(synth.gaussian_probe(m) if blind else np.asarray(c[2], np.complex64))
    fs = [torch.from_numpy(np.asarray(c[3], np.float32)).to(DEV) for c in cases]
    for variant in (0, 1):
        batch = od.ptycho_batch_plan(geoms, fs)
        od.ptycho_batch_set_launch(batch, variant, 0)
        for mb, w0 in zip(batch.members, w0s):
            od.od2p_init(mb, torch.from_numpy(w0).to(DEV))
        assert od.ptycho_plan_get_waves(batch.members[0])[1] >= 1
        batch.iterate(2)
        for i, g in enumerate(geoms):
            alone = od.ptycho_plan(g, fs[i])
            od.ptycho_plan_set_launch(alone, variant, 0)
            od.od2p_init(alone, torch.from_numpy(w0s[i]).to(DEV))
            if g.m == 64:  # the batch runs m = 64 members on the 16 x 4 split
                od.ptycho_plan_set_fft(alone, 2)
            od.od2p_iterate(alone, 2)
            sel = [od.STATE_U, od.STATE_GAMMA, od.STATE_LAMBDA] + (
                [od.STATE_WD, od.STATE_DELTA, od.STATE_W] if g.blind else [])
            for k in sel:
                assert torch.equal(od.od2p_get_state(batch.members[i], k), od.od2p_get_state(alone, k)), (variant, i, k)
            alone.close()
        if variant == 0:  # the blind m = 256 member against the FP64 oracle (two iterations)
            p, (offs, u_true, w, f) = probs[0], cases[0]
            ref = oracle.ADMM(f, w0s[0], offs, p.n, p.n, p.sub_rows, p.sub_cols, p.overlap_px, 0.5, 2.0, 0.5,
                              blind=True, mu=p.mu, gamma=p.gamma)
            ref.iterate(2)
            for k, ko in ((od.STATE_U, oracle.U), (od.STATE_WD, oracle.WD), (od.STATE_W, oracle.W)):
                assert rel_l2(od.od2p_get_state(batch.members[0], k).cpu().numpy(), ref.get(ko)) < 1e-5, k
        batch.close()


def test_batch_with_periodic_members_bitwise():
    """Periodic members (windows wrapping around their images, pairs across the
    boundary) beside a vacuum member: each equals itself iterated alone."""
    specs = [(32, 128, 8, False, True, 51), (64, 192, 16, True, True, 52), (32, 96, 8, True, False, 53)]
    geoms, fs, w0s = [], [], []
    for m, n, step, blind, periodic, seed in specs:
        rng = np.random.default_rng(seed)
        if periodic:
            offs = np.array([(r, c) for r in range(0, n, step) for c in range(0, n, step)], np.int32)
            offs = ((offs + rng.integers(-2, 3, offs.shape)) % n).astype(np.int32)
        else:
            offs = synth.raster_offsets(n, m, step, 1, seed=seed)
        u = (0.5 + 0.5 * rng.random((n, n))) * np.exp(1j * rng.uniform(-1, 1, (n, n)))
        w = synth.make_probe(m).astype(complex)
        f = np.abs(oracle.forward(u, w, offs, periodic=periodic)) ** 2
        geoms.append(od.Geometry(n, n, m, offs, 2, 2, 8, 0.5, 2.0, 0.5, mu=1.0 if blind else 0.0,
                                 gamma=0.1 if blind else 0.0, blind=blind, periodic=periodic))
        fs.append(torch.from_numpy(f.astype(np.float32)).to(DEV))
        w0s.append(synth.gaussian_probe(m) if blind else w.astype(np.complex64))
    batch = od.ptycho_batch_plan(geoms, fs)
    for mb, w0 in zip(batch.members, w0s):
        od.od2p_init(mb, torch.from_numpy(np.asarray(w0, np.complex64)).to(DEV))
    batch.iterate(3)
    for i, g in enumerate(geoms):
        alone = od.ptycho_plan(g, fs[i])
        od.od2p_init(alone, torch.from_numpy(np.asarray(w0s[i], np.complex64)).to(DEV))
        if g.m == 64:  # the batch runs m = 64 members on the 16 x 4 split
            od.ptycho_plan_set_fft(alone, 2)
        od.od2p_iterate(alone, 3)
        for k in (od.STATE_U, od.STATE_GAMMA, od.STATE_LAMBDA):
            assert torch.equal(od.od2p_get_state(batch.members[i], k), od.od2p_get_state(alone, k)), (i, k)
        alone.close()
    batch.close()
