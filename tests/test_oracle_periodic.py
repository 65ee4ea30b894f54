"""Pins of the oracle's periodic-boundary variant (the torus reading of the
decomposition; section 4 names periodic boundaries as the usual alternative to
its vacuum boundary).  Each pin checks it against something other than itself:
the non-periodic oracle where nothing reaches across the boundary, windows cut
with np.roll, translation covariance on the torus, and convergence."""
import numpy as np
import pytest

import oracle


def _rolled_frames(u, w, offs):
    """F(w o S_j u) with S_j the periodic window, cut by rolling the image."""
    m = w.shape[0]
    return np.stack([np.fft.fft2(w * np.roll(u, (-r, -c), axis=(0, 1))[:m, :m], norm="ortho") for r, c in offs])


def _torus_scan(H, W, step, jitter=0, seed=0):
    rng = np.random.default_rng(seed)
    offs = np.array([(r, c) for r in range(0, H, step) for c in range(0, W, step)], np.int32)
    if jitter:
        offs = (offs + rng.integers(-jitter, jitter + 1, offs.shape)) % np.array([H, W])
    return offs.astype(np.int32)


def _image(H, W, seed):
    rng = np.random.default_rng(seed)
    return (0.5 + 0.5 * rng.random((H, W))) * np.exp(1j * rng.uniform(-1, 1, (H, W)))


def _probe(m, seed):
    rng = np.random.default_rng(seed)
    return (0.5 + rng.random((m, m))) * np.exp(1j * rng.uniform(-2, 2, (m, m)))


def test_rolled_windows_match_the_forward_operator_without_wrap():
    """The np.roll windows use the oracle's unitary DFT convention (no frame wraps here)."""
    u, w = _image(16, 16, 1), _probe(4, 2)
    offs = np.array([(0, 0), (3, 5), (12, 12)], np.int32)
    np.testing.assert_allclose(_rolled_frames(u, w, offs), oracle.forward(u, w, offs), atol=1e-13)


@pytest.mark.parametrize("blind", [False, True])
def test_periodic_reduces_to_the_vacuum_oracle_when_nothing_wraps(blind):
    """overlap 0 and a scan inside the image: no rectangle reaches across the
    boundary, so the periodic iterates equal the non-periodic ones exactly."""
    H = W = 24
    m, step = 6, 3
    offs = np.array([(r, c) for r in range(0, H - m + 1, step) for c in range(0, W - m + 1, step)], np.int32)
    u, w = _image(H, W, 3), _probe(m, 4)
    f = np.abs(oracle.forward(u, w, offs)) ** 2 * (1 + 0.05 * np.random.default_rng(5).random((len(offs), m, m)))
    kw = dict(blind=blind, mu=1.0 if blind else 0.0, gamma=0.2 if blind else 0.0)
    a = oracle.ADMM(f, w, offs, H, W, 2, 2, 0, 0.5, 0.3, 0.2, **kw)
    b = oracle.ADMM(f, w, offs, H, W, 2, 2, 0, 0.5, 0.3, 0.2, periodic=True, **kw)
    assert a.P == b.P
    a.iterate(4)
    b.iterate(4)
    for k in (oracle.U, oracle.GAMMA, oracle.LAMBDA, oracle.WD, oracle.W):
        assert np.array_equal(a.get(k), b.get(k)), k
    assert np.array_equal(a.merge(), b.merge())


@pytest.mark.parametrize("grid", [(1, 1), (1, 2), (2, 2), (3, 2)])
def test_periodic_noiseless_truth_is_fixed_point(grid):
    """Intensities of the truth through windows that wrap (cut with np.roll):
    the truth with zero multipliers satisfies every step, across the boundary
    pairs and the self-pairs of a subdomain that reaches around the torus."""
    H, W, m, step = 24, 18, 6, 3
    offs = _torus_scan(H, W, step, jitter=1, seed=6)
    u, w = _image(H, W, 7), _probe(m, 8)
    f = np.abs(_rolled_frames(u, w, offs)) ** 2
    a = oracle.ADMM(f, w, offs, H, W, grid[0], grid[1], 4, 0.5, 0.1, 0.05, u0=u, periodic=True)
    assert a.P > 0  # (1, 1): the single subdomain meets copies of itself
    a.iterate(3)
    np.testing.assert_allclose(a.merge(), u, atol=1e-12)
    assert np.abs(a.get(oracle.GAMMA)).max() < 1e-12
    assert np.abs(a.get(oracle.LAMBDA)).max() < 1e-12
    assert a.metrics()[0] < 1e-12


def test_periodic_wrong_windows_are_not_a_fixed_point():
    """The same check fails for intensities made without the wrap (the pin can fail)."""
    H, W, m, step = 24, 18, 6, 3
    offs = _torus_scan(H, W, step)
    u, w = _image(H, W, 7), _probe(m, 8)
    pad = np.pad(u, ((0, m), (0, m)))  # zeros past the edge instead of the wrapped pixels
    f = np.abs(np.stack([np.fft.fft2(w * pad[r:r + m, c:c + m], norm="ortho") for r, c in offs])) ** 2
    a = oracle.ADMM(f, w, offs, H, W, 2, 2, 4, 0.5, 0.1, 0.05, u0=u, periodic=True)
    a.iterate(1)
    assert a.metrics()[0] > 1e-3


@pytest.mark.parametrize("blind", [False, True])
def test_periodic_covariant_under_a_one_tile_roll(blind):
    """Rolling the scan and the initial image by one core tile relabels the
    subdomains of the torus; after the same iterations the merged image is the
    rolled merged image (FP64, up to the summation order of the pairs)."""
    H, W, m, step, rows, cols = 24, 24, 6, 3, 3, 2
    T = H // rows
    offs = _torus_scan(H, W, step, jitter=1, seed=9)
    u, w = _image(H, W, 10), _probe(m, 11)
    f = np.abs(_rolled_frames(u, w, offs)) ** 2 * (1 + 0.05 * np.random.default_rng(12).random((len(offs), m, m)))
    u0 = _image(H, W, 13)
    kw = dict(periodic=True, blind=blind, mu=1.0 if blind else 0.0, gamma=0.2 if blind else 0.0)
    a = oracle.ADMM(f, w, offs, H, W, rows, cols, 4, 0.5, 0.3, 0.2, u0=u0, **kw)
    offs_t = ((offs + np.array([T, 0])) % np.array([H, W])).astype(np.int32)
    b = oracle.ADMM(f, w, offs_t, H, W, rows, cols, 4, 0.5, 0.3, 0.2, u0=np.roll(u0, T, axis=0), **kw)
    assert a.P == b.P
    a.iterate(5)
    b.iterate(5)
    np.testing.assert_allclose(b.merge(), np.roll(a.merge(), T, axis=0), rtol=0, atol=1e-12)
    if blind:
        np.testing.assert_allclose(b.get(oracle.W), a.get(oracle.W), rtol=0, atol=1e-12)


def test_periodic_noiseless_reconstruction_converges():
    """From u = 1 the residual falls on a periodic scan (blind probe known here)."""
    H, W, m, step = 32, 32, 8, 4
    offs = _torus_scan(H, W, step, jitter=1, seed=14)
    u, w = _image(H, W, 15), _probe(m, 16)
    f = np.abs(_rolled_frames(u, w, offs)) ** 2
    a = oracle.ADMM(f, w, offs, H, W, 2, 2, 4, 0.5, 0.5, 0.3, periodic=True)
    a.iterate(1)
    rf0 = a.metrics()[0]
    a.iterate(60)
    assert a.metrics()[0] < rf0 / 10


def test_periodic_geometry_and_pairs():
    """Extended-coordinate rectangles hold every placed window; each pair (d, e, s)
    is the intersection of Omega_d with Omega_e shifted by s periods, its reverse
    (e, d, -s) is listed, and a placed window's centre lies on the image."""
    H, W, m = 20, 16, 6
    offs = _torus_scan(H, W, 2, jitter=1, seed=17)
    fs, rect, ro = oracle.geometry(H, W, m, offs, 2, 2, 3, periodic=True, placed=True)
    assert np.array_equal(ro % np.array([H, W]), offs)
    for j, (r, c) in enumerate(ro):
        R = rect[fs[j]]
        assert R[0] <= r and r + m <= R[2] and R[1] <= c and c + m <= R[3]
        assert 0 <= 2 * r + m - 1 < 2 * H and 0 <= 2 * c + m - 1 < 2 * W
    pr, sh, prc = oracle.pairs(rect, H, W, periodic=True, shifts=True)
    keys = {(d, e, sr, sc) for (d, e), (sr, sc) in zip(pr, sh)}
    for (d, e), (sr, sc), P in zip(pr, sh, prc):
        A, B = rect[d], rect[e] + np.array([sr * H, sc * W, sr * H, sc * W])
        assert tuple(P) == (max(A[0], B[0]), max(A[1], B[1]), min(A[2], B[2]), min(A[3], B[3]))
        assert (e, d, -sr, -sc) in keys
    # brute force over shifts: every intersecting (d, e, s) is listed
    for d in range(4):
        for e in range(4):
            for sr in range(-3, 4):
                for sc in range(-3, 4):
                    A, B = rect[d], rect[e] + np.array([sr * H, sc * W, sr * H, sc * W])
                    meet = max(A[0], B[0]) < min(A[2], B[2]) and max(A[1], B[1]) < min(A[3], B[3])
                    if meet and not (d == e and sr == 0 and sc == 0):
                        assert (d, e, sr, sc) in keys


def test_periodic_forward_equals_rolled_windows_and_adjoint_identity():
    """Periodic A: frames equal windows cut with np.roll; <A u, y> = <u, A^* y>;
    without wrapping offsets it equals the vacuum operator."""
    rng = np.random.default_rng(18)
    H, W, m = 20, 14, 6
    offs = np.array([(18, 11), (0, 0), (7, 12), (15, 3)], np.int32)
    u, w = _image(H, W, 19), _probe(m, 20)
    A = oracle.forward(u, w, offs, periodic=True)
    np.testing.assert_allclose(A, _rolled_frames(u, w, offs), atol=1e-13)
    y = rng.standard_normal(A.shape) + 1j * rng.standard_normal(A.shape)
    lhs = np.vdot(y, A)
    rhs = np.vdot(oracle.adjoint(y, w, offs, H, W, periodic=True), u)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    inside = np.array([(0, 0), (7, 5), (14, 8)], np.int32)
    np.testing.assert_array_equal(oracle.forward(u, w, inside, periodic=True), oracle.forward(u, w, inside))


def test_periodic_loss_gradient_finite_differences():
    """Periodic loss: the u- and w-gradients against central differences (FP64)."""
    rng = np.random.default_rng(21)
    H, W, m = 12, 10, 4
    offs = np.array([(10, 8), (3, 9), (0, 0), (6, 4)], np.int32)
    u, w = _image(H, W, 22), _probe(m, 23)
    f = np.abs(_rolled_frames(_image(H, W, 24), w, offs)) ** 2
    loss, gu, gw = oracle.loss_grad(u, w, offs, f, 0.5, periodic=True)
    h = 1e-6
    for _ in range(6):
        R, C = rng.integers(0, H), rng.integers(0, W)
        for d in (1.0, 1j):
            up, um = u.copy(), u.copy()
            up[R, C] += h * d
            um[R, C] -= h * d
            fd = (oracle.loss_grad(up, w, offs, f, 0.5, periodic=True)[0] -
                  oracle.loss_grad(um, w, offs, f, 0.5, periodic=True)[0]) / (2 * h)
            # the gradient is d loss / d Re u + i d loss / d Im u
            want = gu[R, C].real if d == 1.0 else gu[R, C].imag
            assert abs(fd - want) < 1e-5 * max(1.0, abs(want)), (R, C, d, fd, want)
    k = (1, 2)
    wp, wm = w.copy(), w.copy()
    wp[k] += h
    wm[k] -= h
    fd = (oracle.loss_grad(u, wp, offs, f, 0.5, periodic=True)[0] -
          oracle.loss_grad(u, wm, offs, f, 0.5, periodic=True)[0]) / (2 * h)
    assert abs(fd - gw[k].real) < 1e-5 * max(1.0, abs(fd))
