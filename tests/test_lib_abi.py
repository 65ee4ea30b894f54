"""The C ABI library loads without a GPU and exports every symbol its header declares."""
import ctypes
import os
import re

import pytest

from paper_2011_00162_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "od2p.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["ptycho_plan", "ptycho_forward", "stagm_prox", "overlap_add", "od2p_iterate",
                     "probe_update", "od2p_init", "stagm_loss_grad", "ptycho_plan_destroy"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, f"binding lacks {n}"


def test_abi_version_and_argument_errors(lib):
    assert lib.ptycho_abi_version() == 3
    # argument checks return before any device work
    assert lib.ptycho_plan(None, None, None, None) == _lib.ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.ptycho_plan(ctypes.byref(h), None, None, None) == _lib.ERR_INVALID_ARG
    assert b"NULL" in lib.ptycho_last_error()
    assert lib.stagm_prox(None, None, None, -1, 0.5, 0.1, None) == _lib.ERR_INVALID_ARG
    assert lib.stagm_prox(None, None, None, 0, 1.5, 0.1, None) == _lib.ERR_INVALID_ARG
    assert lib.stagm_prox(None, None, None, 0, 0.5, 0.1, None) == _lib.OK
    assert lib.od2p_iterate(None, 1, None) == _lib.ERR_INVALID_ARG
    assert lib.ptycho_plan_set_launch(None, 0, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.ptycho_probe_init(None, None, None) == _lib.ERR_INVALID_ARG
    assert lib.od2p_set_penalties(None, 1.0, 1.0, None) == _lib.ERR_INVALID_ARG
    assert lib.od2p_consensus_residual(None, None, None) == _lib.ERR_INVALID_ARG
    assert lib.od2p_snr(None, None, None, None, None) == _lib.ERR_INVALID_ARG
    assert lib.od2p_operator_norms(None, None, None) == _lib.ERR_INVALID_ARG
    assert lib.ptycho_peak_probe(2, 1, 1, None, None) == _lib.ERR_INVALID_ARG
    assert lib.od2p_iterate_until(None, 1e-5, 10, None, None, None) == _lib.ERR_INVALID_ARG
    assert lib.od2p_gamma_snapshot(None, None) == _lib.ERR_INVALID_ARG
    assert lib.ptycho_plan_set_fft(None, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.ptycho_plan_get_fft(None, None) == _lib.ERR_INVALID_ARG
    assert lib.od2p_frame_residual(None, None, None) == _lib.ERR_INVALID_ARG
    assert lib.ptycho_plan_get_launch(None, None, None, None) == _lib.ERR_INVALID_ARG
    assert lib.ptycho_batch_set_launch(None, 0, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.ptycho_batch_get_launch(None, None, None) == _lib.ERR_INVALID_ARG
    assert lib.ptycho_plan_destroy(None) == _lib.OK


def test_plan_rejects_bad_geometry_before_device_work(lib):
    import numpy as np
    offs = np.array([[0, 0], [0, 70]], np.int32)  # second window leaves a 64-wide image
    f = ctypes.c_void_p(1)  # never dereferenced: validation fails first
    for m, eps, code in [(64, 0.5, _lib.ERR_INVALID_ARG), (40, 0.5, _lib.ERR_UNSUPPORTED),
                         (16, 1.5, _lib.ERR_INVALID_ARG)]:
        g = _lib.Geometry(64, 64, m, 2, offs.ctypes.data, 1, 1, 0, eps, 0.1, 0.1, 0, 0, 0, None)
        h = ctypes.c_void_p()
        assert lib.ptycho_plan(ctypes.byref(h), ctypes.byref(g), f, None) == code
        assert not h.value


def test_decomposition_on_the_host_equals_the_oracle():
    """ptycho_decompose runs on the host (no device work): bit-exact against the
    oracle's decomposition, so ranks can split a problem before any plan exists."""
    import numpy as np

    import oracle
    import paper_2011_00162_gb300 as od
    from paper_2011_00162_gb300 import synth
    for n, m, step, jit, grid, ov in [(512, 64, 16, 2, (4, 4), 16), (300, 32, 12, 3, (3, 5), 0),
                                      (96, 16, 6, 1, (3, 3), 8), (4096, 256, 48, 4, (8, 8), 64)]:
        offs = synth.raster_offsets(n, m, step, jit, seed=5)
        fs, rect = od.ptycho_decompose(od.Geometry(n, n, m, offs, grid[0], grid[1], ov))
        fo, ro = oracle.geometry(n, n, m, offs, grid[0], grid[1], ov)
        assert np.array_equal(fs, fo) and np.array_equal(rect, ro)


def test_periodic_decomposition_on_the_host_equals_the_oracle():
    """Periodic boundaries: the host decomposition (extended-coordinate
    rectangles, frames placed at the copy whose centre lies on the image) is
    bit-exact against the oracle's, and a rectangle reaching a period beyond the
    image is refused."""
    import numpy as np

    import oracle
    import paper_2011_00162_gb300 as od
    rng = np.random.default_rng(8)
    for n, m, step, grid, ov in [(96, 16, 6, (3, 3), 8), (128, 32, 8, (2, 4), 4), (64, 16, 4, (1, 1), 6),
                                 (256, 64, 16, (4, 4), 16)]:
        offs = np.array([(r, c) for r in range(0, n, step) for c in range(0, n, step)], np.int32)
        offs = ((offs + rng.integers(-2, 3, offs.shape)) % n).astype(np.int32)
        fs, rect = od.ptycho_decompose(od.Geometry(n, n, m, offs, grid[0], grid[1], ov, periodic=True))
        fo, ro = oracle.geometry(n, n, m, offs, grid[0], grid[1], ov, periodic=True)
        assert np.array_equal(fs, fo) and np.array_equal(rect, ro), (n, m, grid)
    # offsets anywhere on the torus are accepted only with periodic boundaries
    offs = np.array([[90, 90]], np.int32)
    with pytest.raises(od.PtychoError):
        od.ptycho_decompose(od.Geometry(96, 96, 16, offs, 1, 1, 0))
    od.ptycho_decompose(od.Geometry(96, 96, 16, offs, 1, 1, 0, periodic=True))
    # a 1 x 1 grid with a wide overlap reaches more than a period beyond the image
    with pytest.raises(od.PtychoError):
        od.ptycho_decompose(od.Geometry(32, 32, 16, offs % 32, 1, 1, 70, periodic=True))


def test_decomposition_fuzz_against_the_oracle():
    """Random geometries (image sides, probe sides up to the image, steps, jitter,
    grids up to 5 x 5, overlaps), vacuum and periodic boundaries: the host
    decomposition equals the oracle's bit for bit, and both refuse the same
    inputs."""
    import numpy as np

    import oracle
    import paper_2011_00162_gb300 as od
    rng = np.random.default_rng(2024)
    checked = 0
    for _ in range(120):
        m = int(rng.choice([16, 32, 48, 64]))
        n = int(rng.integers(m, 4 * m + 1))
        step = int(rng.integers(max(1, m // 8), m + 1))
        rows, cols = int(rng.integers(1, 6)), int(rng.integers(1, 6))
        ov = int(rng.integers(0, 2 * m))
        periodic = bool(rng.integers(0, 2))
        if periodic:
            offs = np.array([(r, c) for r in range(0, n, step) for c in range(0, n, step)], np.int32)
            offs = ((offs + rng.integers(-3, 4, offs.shape)) % n).astype(np.int32)
        else:
            lim = n - m
            offs = np.array([(r, c) for r in range(0, lim + 1, step) for c in range(0, lim + 1, step)], np.int32)
            offs = np.clip(offs + rng.integers(-3, 4, offs.shape), 0, lim).astype(np.int32)
        g = od.Geometry(n, n, m, offs, rows, cols, ov, periodic=periodic)
        try:
            fo, ro = oracle.geometry(n, n, m, offs, rows, cols, ov, periodic=periodic)
        except ValueError:
            with pytest.raises(od.PtychoError):
                od.ptycho_decompose(g)
            continue
        fs, rect = od.ptycho_decompose(g)
        assert np.array_equal(fs, fo) and np.array_equal(rect, ro), (n, m, step, rows, cols, ov, periodic)
        checked += 1
    assert checked > 60
