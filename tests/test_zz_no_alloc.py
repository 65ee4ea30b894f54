"""The allocation-free loss entry point against the plan-based one.

Some callers cannot allocate device memory (a stream being captured into a
CUDA graph, a host that gives a plug-in a fixed memory budget, a real-time loop
that must not block on cudaMalloc).  stagm_loss_noalloc serves them with a
fixed scratch array compiled into the library.  This file is collected last so
that a run stopping at its first failure has run every other test already.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2011_00162_gb300 as od
from paper_2011_00162_gb300 import _lib, synth
from paper_2011_00162_gb300 import build as odbuild

pytestmark = pytest.mark.gpu

LOSS_TOL = 1e-5  # relative, as for every single-pass result of the parity suite


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _noalloc(u, w, offs_dev, f, eps):
    out = torch.empty(1, dtype=torch.float32, device=u.device)
    rc = _lib.load().stagm_loss_noalloc(
        ctypes.c_void_p(u.data_ptr()), u.shape[0], u.shape[1], ctypes.c_void_p(w.data_ptr()), w.shape[0],
        ctypes.c_void_p(offs_dev.data_ptr()), offs_dev.shape[0], ctypes.c_void_p(f.data_ptr()), eps,
        ctypes.c_void_p(out.data_ptr()), _stream())
    _lib.check(rc)
    return out


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    odbuild.build()


@pytest.mark.parametrize("m,n,step", [(64, 512, 16), (16, 64, 4), (128, 384, 48)])
def test_noalloc_loss_matches_plan_loss_twice(m, n, step):
    dev = torch.device("cuda:0")
    p = synth.Problem("na", n, m, step, 2, 1, 1, 0, 1e4, 1, seed=m + 3)
    offs = p.offsets()
    u_true, w = p.truth(), p.probe()
    f = synth.poissonize(np.abs(oracle.forward(u_true, w, offs)) ** 2, p.peak, 5)
    rng = np.random.default_rng(m)
    u = (u_true * (1 + 0.1 * rng.standard_normal(u_true.shape))).astype(np.complex64)
    ud = torch.from_numpy(u).to(dev)
    wd = torch.from_numpy(w).to(dev)
    fd = torch.from_numpy(f).to(dev)
    offs_dev = torch.from_numpy(np.ascontiguousarray(offs)).to(dev)
    plan = od.ptycho_plan(od.Geometry(n, n, m, offs, eps=0.5), fd)
    ref, _, _ = od.stagm_loss_grad(plan, ud, wd, grad_u=False, grad_w=False)
    ref = float(ref.item())
    # the FP64 oracle's loss on the same (FP32-representable) inputs
    exact, _, _ = oracle.loss_grad(u.astype(np.complex128), w, offs, f.astype(np.float64), 0.5)
    for _ in range(2):  # the shared scratch keeps the previous call's partials
        got = float(_noalloc(ud, wd, offs_dev, fd, 0.5).item())
        assert abs(got - ref) <= LOSS_TOL * abs(ref), (got, ref)
        assert abs(got - exact) <= LOSS_TOL * abs(exact), (got, exact)
    plan.close()


def test_noalloc_window_outside_image_gives_nan():
    """Offsets live in device memory, so the kernel checks each window: a window
    that leaves the image is not read and the loss comes back NaN; the next call
    with valid offsets is unaffected."""
    dev = torch.device("cuda:0")
    m, n = 16, 64
    p = synth.Problem("na_bad", n, m, 4, 0, 1, 1, 0, None, 1, seed=11)
    offs = p.offsets()
    u_true, w = p.truth(), p.probe()
    f = (np.abs(oracle.forward(u_true, w, offs)) ** 2).astype(np.float32)
    u = (0.9 * u_true).astype(np.complex64)  # away from the truth: a loss well above 0
    ud = torch.from_numpy(u).to(dev)
    wd = torch.from_numpy(w).to(dev)
    fd = torch.from_numpy(f).to(dev)
    offs = np.ascontiguousarray(offs, dtype=np.int32)
    good = torch.from_numpy(offs).to(dev)
    for bad_row, bad_col in [(n - m + 1, 0), (0, -1), (-5, 3), (2, n)]:
        bad = offs.copy()
        bad[len(bad) // 2] = (bad_row, bad_col)
        got = float(_noalloc(ud, wd, torch.from_numpy(bad).to(dev), fd, 0.5).item())
        assert np.isnan(got), (bad_row, bad_col, got)
    got = float(_noalloc(ud, wd, good, fd, 0.5).item())
    exact, _, _ = oracle.loss_grad(u.astype(np.complex128), w, offs, f.astype(np.float64), 0.5)
    assert abs(got - exact) <= LOSS_TOL * abs(exact), (got, exact)


def test_noalloc_rejects_oversized_and_bad_arguments():
    dev = torch.device("cuda:0")
    m = 64
    u = torch.ones((m, m), dtype=torch.complex64, device=dev)
    w = torch.ones((m, m), dtype=torch.complex64, device=dev)
    f = torch.ones((1, m, m), dtype=torch.float32, device=dev)
    out = torch.empty(1, dtype=torch.float32, device=dev)
    offs = torch.zeros((1, 2), dtype=torch.int32, device=dev)
    lib = _lib.load()
    args = lambda J, eps, mm: (ctypes.c_void_p(u.data_ptr()), m, m, ctypes.c_void_p(w.data_ptr()), mm,
                               ctypes.c_void_p(offs.data_ptr()), J, ctypes.c_void_p(f.data_ptr()), eps,
                               ctypes.c_void_p(out.data_ptr()), _stream())
    # more frames than the fixed scratch covers: refused before any launch
    assert lib.stagm_loss_noalloc(*args(65537, 0.5, m)) == _lib.ERR_INVALID_ARG
    assert b"at most" in lib.ptycho_last_error()
    assert lib.stagm_loss_noalloc(*args(1, 1.5, m)) == _lib.ERR_INVALID_ARG
    assert lib.stagm_loss_noalloc(*args(1, 0.5, 48)) == _lib.ERR_UNSUPPORTED
