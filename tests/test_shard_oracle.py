"""Subdomain sharding of one reconstruction over CPU ranks (gloo).

Each rank runs the FP64 oracle on its own contiguous block of subdomains
(multi.partition_subdomains), keeps halo copies of the others, and exchanges
the overlap strips of u and Lambda (and, blind, W_d and Delta_d) with the
other ranks before every iteration (multi.HaloSchedule, multi.exchange_halos).
After the run, every owned value must equal the single-process oracle's bit
for bit: the ranks compute exactly the undivided iteration (section 3.1, the
subdomain problems being coupled only through their overlaps).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2011_00162_gb300 import multi, synth

N_IT = 6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(blind, periodic=False):
    p = synth.Problem("shard", 96, 16, 6, 1, 3, 3, 8, 1e3, 1, eta=2.0, r=0.5, seed=17)
    offs = p.offsets()
    if periodic:  # a raster over the whole torus: windows wrap around the image
        offs = np.array([(r, c) for r in range(0, p.n, p.step) for c in range(0, p.n, p.step)], np.int32)
        offs = ((offs + np.random.default_rng(3).integers(-1, 2, offs.shape)) % p.n).astype(np.int32)
    u, w = p.truth(), p.probe()
    f = synth.poissonize(np.abs(oracle.forward(u, w, offs, periodic=periodic)) ** 2, p.peak, 5).astype(np.float64)
    w0 = synth.gaussian_probe(p.m) if blind else w
    return p, offs, f, w0


def _admm(p, offs, f, w0, blind, periodic=False):
    return oracle.ADMM(f, w0, offs, p.n, p.n, p.sub_rows, p.sub_cols, p.overlap_px, p.eps, p.eta, p.r,
                       blind=blind, mu=1.0 if blind else 0.0, gamma=0.1 if blind else 0.0, periodic=periodic)


SEL = {"u": oracle.U, "lam": oracle.LAMBDA, "W": oracle.WD, "Delta": oracle.DELTA}


def _worker(rank, world, port, blind, periodic, out):
    torch.set_num_threads(1)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p, offs, f, w0 = _case(blind, periodic)
    a = _admm(p, offs, f, w0, blind, periodic)
    fs, rect = oracle.geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px, periodic=periodic)
    pr, prc = oracle.pairs(rect, p.n, p.n, periodic=periodic)
    owner = multi.partition_subdomains(fs, len(rect), world)
    a.set_owned([1 if o == rank else 0 for o in owner])
    sched = multi.HaloSchedule(rect, pr, prc, owner, rank, p.m, blind)
    names = ["u", "lam"] + (["W", "Delta"] if blind else [])
    for _ in range(N_IT):
        arrays = {k: torch.from_numpy(a.get(SEL[k]).copy()) for k in names}
        multi.exchange_halos(sched, arrays)
        for k in names:
            a.set(SEL[k], arrays[k].numpy())
        a.iterate(1)
    res = {"owner": owner, "U": a.get(oracle.U), "LAMBDA": a.get(oracle.LAMBDA), "GAMMA": a.get(oracle.GAMMA),
           "W": a.get(oracle.W), "WD": a.get(oracle.WD), "DELTA": a.get(oracle.DELTA),
           "sizes": {q: multi.HaloSchedule.size(s) for q, s in sched.send.items()}}
    got = [None] * world
    dist.all_gather_object(got, res)
    if rank == 0:
        out.put(got)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("blind", [False, True])
@pytest.mark.parametrize("world", [2, 4])
def test_sharded_oracle_equals_single_process(world, blind, periodic):
    p, offs, f, w0 = _case(blind, periodic)
    ref = _admm(p, offs, f, w0, blind, periodic)
    ref.iterate(N_IT)
    fs, rect = oracle.geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px, periodic=periodic)
    pr, prc = oracle.pairs(rect, p.n, p.n, periodic=periodic)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, blind, periodic, q)) for r in range(world)]
    for pc in procs:
        pc.start()
    got = q.get(timeout=300)
    for pc in procs:
        pc.join(timeout=60)
        assert pc.exitcode == 0
    owner = got[0]["owner"]
    assert sorted(set(owner)) == list(range(world))          # every rank owns a block
    assert owner == sorted(owner)                              # contiguous blocks
    sched = multi.HaloSchedule(rect, pr, prc, owner, 0, p.m, blind)
    u_ref, lam_ref, gam_ref = ref.get(oracle.U), ref.get(oracle.LAMBDA), ref.get(oracle.GAMMA)
    mm = p.m * p.m
    for r, res in enumerate(got):
        for d in range(len(rect)):
            if owner[d] != r:
                continue
            sl = slice(sched.u_off[d], sched.u_off[d + 1])
            assert np.array_equal(res["U"][sl], u_ref[sl]), (r, d)
            if blind:
                assert np.array_equal(res["WD"][d * mm:(d + 1) * mm], ref.get(oracle.WD)[d * mm:(d + 1) * mm])
                assert np.array_equal(res["DELTA"][d * mm:(d + 1) * mm], ref.get(oracle.DELTA)[d * mm:(d + 1) * mm])
        for k, (d, e) in enumerate(pr):
            if owner[d] == r:
                sl = slice(sched.lam_off[k], sched.lam_off[k + 1])
                assert np.array_equal(res["LAMBDA"][sl], lam_ref[sl]), (r, d, e)
        for j in range(len(offs)):
            if owner[fs[j]] == r:
                assert np.array_equal(res["GAMMA"][j * mm:(j + 1) * mm], gam_ref[j * mm:(j + 1) * mm])
        if blind:
            assert np.array_equal(res["W"], ref.get(oracle.W))


def test_partition_and_schedule_host_logic():
    # balanced contiguous blocks, every rank non-empty
    assert multi.partition_subdomains([0, 0, 1, 1, 2, 2, 3, 3, 3], 4, 2) == [0, 0, 1, 1]
    assert multi.partition_subdomains([0] * 8 + [1, 2, 3], 4, 4) == [0, 1, 2, 3]
    assert multi.partition_subdomains(list(range(16)) * 3, 16, 3) == [0] * 5 + [1] * 6 + [2] * 5
    # the messages of a pair of ranks mirror each other
    p, offs, f, w0 = _case(False)
    fs, rect = oracle.geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px)
    pr, prc = oracle.pairs(rect)
    owner = multi.partition_subdomains(fs, len(rect), 3)
    s = [multi.HaloSchedule(rect, pr, prc, owner, r, p.m, False) for r in range(3)]
    for a in range(3):
        for b in range(3):
            if a != b:
                assert s[a].send[b] == s[b].recv[a]
    # a round trip through pack / unpack restores exactly the strips and nothing else
    rng = np.random.default_rng(0)
    arrays = {"u": rng.standard_normal(s[0].u_off[-1]) + 0j, "lam": rng.standard_normal(s[0].lam_off[-1]) + 0j}
    msg = s[0].pack(1, arrays)
    blank = {k: np.zeros_like(v) for k, v in arrays.items()}
    s[1].unpack(0, msg, blank)
    touched = {k: blank[k] != 0 for k in blank}
    for k in arrays:
        assert np.array_equal(blank[k][touched[k]], arrays[k][touched[k]])
    # (strips of one u_e toward two neighbours may share corner pixels)
    assert 0 < touched["u"].sum() + touched["lam"].sum() <= msg.size
    assert touched["lam"].sum() == sum(rows * cols for name, _, _, rows, cols in s[0].send[1] if name == "lam")
