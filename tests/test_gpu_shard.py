"""Shard plans on one GPU: a reconstruction split over 2 or 4 shards (the
contiguous subdomain blocks of multi.partition_subdomains), halos exchanged
between iterations by the library's pack / unpack calls, equals the whole plan
bit for bit in every owned value.  The shards run one after another on one
stream (none waits on another); the multi-GPU exchange itself (NCCL between
ranks, multi.exchange_shard_halos) is not run here."""
import numpy as np
import pytest
import torch

import oracle
import paper_2011_00162_gb300 as od
from paper_2011_00162_gb300 import multi, synth
from paper_2011_00162_gb300 import build as odbuild

from _cases import make_case

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    odbuild.build()


CASES = [("nonblind_m64_4x4", 384, 64, 16, 4, False, False), ("blind_m32_3x3", 160, 32, 8, 3, True, False),
         ("blind_m256_2x2", 512, 256, 64, 2, True, False), ("nonblind_m48_3x2", 192, 48, 12, 3, False, False),
         ("periodic_blind_m32_3x3", 160, 32, 8, 3, True, True), ("periodic_nonblind_m64_2x2", 256, 64, 16, 2, False, True)]


@pytest.mark.parametrize("name,n,m,step,grid,blind,periodic", CASES)
@pytest.mark.parametrize("world", [2, 4])
def test_shards_equal_whole_plan(name, n, m, step, grid, blind, periodic, world):
    p = synth.Problem(name, n, m, step, 1, grid, grid - (1 if name.endswith("3x2") else 0), 8, 1e4, 1,
                      eta=2.0, r=0.5, blind=blind, mu=1.0 if blind else 0.0, gamma=0.1 if blind else 0.0, seed=41)
    offs, u_true, w, f = make_case(p)
    if periodic:  # a raster over the whole torus: windows wrap around the image
        offs = np.array([(r, c) for r in range(0, n, step) for c in range(0, n, step)], np.int32)
        offs = ((offs + np.random.default_rng(4).integers(-1, 2, offs.shape)) % n).astype(np.int32)
        f = np.abs(oracle.forward(u_true, w, offs, periodic=True)) ** 2
    w0 = synth.gaussian_probe(m) if blind else w
    g = od.Geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px, p.eps, p.eta, p.r, mu=p.mu,
                    gamma=p.gamma, blind=blind, periodic=periodic)
    fs, rect = od.ptycho_decompose(g)
    D = len(rect)
    if world > D:
        pytest.skip("more ranks than subdomains")
    owner = multi.partition_subdomains(fs, D, world)
    f_t = torch.from_numpy(np.asarray(f, np.float32)).to(DEV)
    whole = od.ptycho_plan(g, f_t)
    od.od2p_init(whole, torch.from_numpy(w0.astype(np.complex64)).to(DEV))
    shards = []
    for r in range(world):
        sel = np.flatnonzero(np.asarray(owner)[fs] == r)
        sh = od.ptycho_plan_shard(g, owner, r, f_t[torch.from_numpy(sel).to(DEV)].contiguous())
        assert np.array_equal(od.ptycho_plan_frames(sh), sel)
        od.od2p_init(sh, torch.from_numpy(w0.astype(np.complex64)).to(DEV))
        shards.append(sh)
    # the library's messages follow the same schedule as multi.HaloSchedule
    _, _, pr, prc = whole.layout()
    for r in range(world):
        hs = multi.HaloSchedule(rect, pr, prc, owner, r, m, blind)
        for q in range(world):
            if q != r:
                assert od.od2p_halo_size(shards[r], q) == (multi.HaloSchedule.size(hs.send[q]),
                                                          multi.HaloSchedule.size(hs.recv[q]))
    n_it = 4
    for _ in range(n_it):
        multi.exchange_local(shards)
        for sh in shards:
            od.od2p_iterate(sh, 1)
    od.od2p_iterate(whole, n_it)
    # cross-check one message against the Python schedule applied to the shard's state
    r0, q0 = 0, 1
    hs = multi.HaloSchedule(rect, pr, prc, owner, r0, m, blind)
    arrays = {"u": od.od2p_get_state(shards[r0], od.STATE_U), "lam": od.od2p_get_state(shards[r0], od.STATE_LAMBDA)}
    if blind:
        arrays["W"] = od.od2p_get_state(shards[r0], od.STATE_WD)
        arrays["Delta"] = od.od2p_get_state(shards[r0], od.STATE_DELTA)
    assert torch.equal(od.od2p_halo_pack(shards[r0], q0), hs.pack(q0, arrays))
    # every owned value equals the whole plan's
    u_off = [0]
    for r0_, c0_, r1_, c1_ in rect:
        u_off.append(u_off[-1] + (r1_ - r0_) * (c1_ - c0_))
    lam_off = [0]
    for a in prc:
        lam_off.append(lam_off[-1] + (a[2] - a[0]) * (a[3] - a[1]))
    U, LAM, GAM = (od.od2p_get_state(whole, k) for k in (od.STATE_U, od.STATE_LAMBDA, od.STATE_GAMMA))
    mm = m * m
    for r, sh in enumerate(shards):
        u_s, lam_s, gam_s = (od.od2p_get_state(sh, k) for k in (od.STATE_U, od.STATE_LAMBDA, od.STATE_GAMMA))
        for d in range(D):
            if owner[d] == r:
                assert torch.equal(u_s[u_off[d]:u_off[d + 1]], U[u_off[d]:u_off[d + 1]]), (r, d)
        for k, (d, e) in enumerate(pr):
            if owner[d] == r:
                assert torch.equal(lam_s[lam_off[k]:lam_off[k + 1]], LAM[lam_off[k]:lam_off[k + 1]]), (r, d, e)
        sel = od.ptycho_plan_frames(sh)
        G = GAM.reshape(-1, mm)[torch.from_numpy(sel).to(DEV)].reshape(-1)
        assert torch.equal(gam_s, G)
        if blind:
            Wd_w, De_w = od.od2p_get_state(whole, od.STATE_WD), od.od2p_get_state(whole, od.STATE_DELTA)
            Wd_s, De_s = od.od2p_get_state(sh, od.STATE_WD), od.od2p_get_state(sh, od.STATE_DELTA)
            for d in range(D):
                if owner[d] == r:
                    assert torch.equal(Wd_s[d * mm:(d + 1) * mm], Wd_w[d * mm:(d + 1) * mm])
                    assert torch.equal(De_s[d * mm:(d + 1) * mm], De_w[d * mm:(d + 1) * mm])
            assert torch.equal(od.od2p_get_state(sh, od.STATE_W), od.od2p_get_state(whole, od.STATE_W))
    for sh in shards:
        sh.close()
    whole.close()


def test_shard_argument_errors():
    p = synth.Problem("e", 160, 32, 8, 1, 2, 2, 8, 1e4, 1, seed=3)
    offs, u_true, w, f = make_case(p)
    g = od.Geometry(p.n, p.n, p.m, offs, 2, 2, 8)
    fs, rect = od.ptycho_decompose(g)
    f_t = torch.from_numpy(np.asarray(f, np.float32)).to(DEV)
    with pytest.raises((ValueError, od.PtychoError)):  # rank 3 owns nothing
        od.ptycho_plan_shard(g, [0, 0, 1, 1], 3, f_t[:1].contiguous())
    # the C ABI refuses it too
    import ctypes
    from paper_2011_00162_gb300 import _lib
    gs, keep = od.api._geometry_struct(g)
    own = np.array([0, 0, 1, 1], np.int32)
    h = ctypes.c_void_p()
    rc = _lib.load().ptycho_plan_shard(ctypes.byref(h), ctypes.byref(gs), own.ctypes.data, 3,
                                        ctypes.c_void_p(f_t.data_ptr()), None)
    assert rc == _lib.ERR_INVALID_ARG and not h.value
    whole = od.ptycho_plan(g, f_t)
    with pytest.raises(od.PtychoError) as e:
        od.od2p_halo_size(whole, 1)
    assert e.value.code == 6  # PTYCHO_ERR_STATE: not a shard
    owner = [0, 0, 1, 1]
    sel = np.flatnonzero(np.asarray(owner)[fs] == 0)
    sh = od.ptycho_plan_shard(g, owner, 0, f_t[torch.from_numpy(sel).to(DEV)].contiguous())
    for bad in (0, 2, -1):
        with pytest.raises(od.PtychoError):
            od.od2p_halo_size(sh, bad)
