"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: each test checks it against an
independent statement -- numpy's FFT, the DFT written as a dense matrix,
brute-force minimisation, finite differences, a dense least-squares solve of
the ADMM subproblem as the paper states it, exact fixed points, or numbers
printed in the paper (tests/golden/paper_geometry.json).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2011_00162_gb300 import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_geometry.json")))
RNG = np.random.default_rng(12345)


def crandn(*shape, rng=RNG):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ----------------------------------------------------------------------------- FFT
@pytest.mark.parametrize("m", [2, 4, 8, 16, 6, 12, 15])
def test_fft_radix2_equals_dft_definition(m):
    x = crandn(m, m)
    np.testing.assert_allclose(oracle.fft2(x), oracle.dft2(x), atol=1e-12)
    np.testing.assert_allclose(oracle.fft2(x, True), oracle.dft2(x, True), atol=1e-12)


@pytest.mark.parametrize("m", [16, 32, 64, 128, 48, 80, 96])
def test_fft_matches_numpy_unitary(m):
    x = crandn(m, m)
    np.testing.assert_allclose(oracle.fft2(x), np.fft.fft2(x, norm="ortho"), atol=1e-11)
    np.testing.assert_allclose(oracle.fft2(x, True), np.fft.ifft2(x, norm="ortho"), atol=1e-11)


def test_fft_parseval_inverse_delta():
    m = 32
    x = crandn(m, m)
    X = oracle.fft2(x)
    assert abs(np.linalg.norm(X) - np.linalg.norm(x)) < 1e-10 * np.linalg.norm(x)
    np.testing.assert_allclose(oracle.fft2(X, True), x, atol=1e-12)
    d = np.zeros((m, m), complex)
    d[0, 0] = 1.0
    np.testing.assert_allclose(oracle.fft2(d), np.full((m, m), 1.0 / m), atol=1e-15)


# ----------------------------------------------------------------------------- ST-AGM
@pytest.mark.parametrize("eps", [0.1, 0.5, 0.9])
def test_stagm_continuous_and_reduces_to_agm(eps):
    b = 2.3
    edge = eps * math.sqrt(b)
    th = np.exp(1j * 0.7)
    lo, hi = oracle.stagm_g(np.array([(edge - 1e-10) * th, (edge + 1e-10) * th]), b, eps)
    assert abs(lo - hi) < 1e-8
    # outside the truncation disk g is the amplitude-Gaussian metric 1/2 (|x| - sqrt b)^2
    x = crandn(200) * 3
    x = x[np.abs(x) >= edge]
    np.testing.assert_allclose(oracle.stagm_g(x, b, eps), 0.5 * (np.abs(x) - math.sqrt(b)) ** 2)
    # eps -> 0: ST-AGM is AGM everywhere
    x = crandn(200)
    np.testing.assert_allclose(oracle.stagm_g(x, b, 1e-12), 0.5 * (np.abs(x) - math.sqrt(b)) ** 2,
                               atol=1e-10)


@pytest.mark.parametrize("eps", [0.1, 0.5, 0.9])
def test_stagm_minimiser_unchanged(eps):
    """Section 2.2: for eps in (0, 1) the minimiser |x| = sqrt(b) does not move."""
    b = 1.7
    rho = np.linspace(0, 3, 300001)
    g = oracle.stagm_g(rho.astype(complex), b, eps)
    assert abs(rho[np.argmin(g)] - math.sqrt(b)) < 2e-5
    assert g.min() < 1e-12


@pytest.mark.parametrize("eps", [0.2, 0.5, 0.8])
def test_stagm_gradient_finite_differences(eps):
    b = np.abs(RNG.standard_normal(400)) + 0.2
    x = crandn(400) * np.sqrt(b) * 0.9  # both regions K1 and K2
    h = 1e-6
    fd = (oracle.stagm_g(x + h, b, eps) - oracle.stagm_g(x - h, b, eps)) / (2 * h) + 1j * (
        oracle.stagm_g(x + 1j * h, b, eps) - oracle.stagm_g(x - 1j * h, b, eps)) / (2 * h)
    far = np.abs(np.abs(x) - eps * np.sqrt(b)) > 1e-4
    np.testing.assert_allclose(oracle.stagm_grad(x, b, eps)[far], fd[far], atol=2e-7)


@pytest.mark.parametrize("eps", GOLDEN["lipschitz"]["eps"])
def test_stagm_gradient_lipschitz_bound(eps):
    """Lemma 2.1: |grad g(x1) - grad g(x2)| <= (2/eps - 1) |x1 - x2|."""
    L = 2.0 / eps - 1.0
    b = 1.0
    x1 = crandn(20000) * 0.8
    x2 = x1 + crandn(20000) * RNG.choice([1e-3, 1e-1, 1.0], 20000)
    ratio = np.abs(oracle.stagm_grad(x1, b, eps) - oracle.stagm_grad(x2, b, eps)) / np.abs(x1 - x2)
    assert ratio.max() <= L + 1e-9
    # the bound is attained up to its slack: the exact constant is max(1, 1/eps - 1)
    assert ratio.max() >= 0.95 * max(1.0, 1.0 / eps - 1.0)


def _prox_objective(z, y, f, eps, lam):
    return oracle.stagm_g(z, f, eps) + 0.5 * lam * np.abs(z - y) ** 2


@pytest.mark.parametrize("eps", [0.1, 0.5, 0.9])
@pytest.mark.parametrize("lam", [0.05, 0.1, 1.0, 2.0, 20.0])
def test_stagm_prox_brute_force(eps, lam):
    """eq. (Prox_sol) against brute-force minimisation over the complex plane."""
    rng = np.random.default_rng(int(eps * 100 + lam * 10))
    for _ in range(40):
        f = float(rng.choice([0.0, 1e-3, 0.5, 1.0, 4.0]))
        y = complex(rng.standard_normal() * 2, rng.standard_normal() * 2) * rng.choice([1e-2, 0.3, 1.0])
        z = oracle.stagm_prox(np.array([y]), f, eps, lam)[0]
        # brute force in polar coordinates around the origin
        R = 1.5 * (abs(y) + math.sqrt(f)) + 0.1
        rho = np.linspace(0, R, 801)
        th = np.linspace(-math.pi, math.pi, 721)
        Z = rho[:, None] * np.exp(1j * th[None, :])
        obj = _prox_objective(Z, y, f, eps, lam)
        zb = Z.flat[np.argmin(obj)]
        ob = obj.min()
        oc = _prox_objective(np.array([z]), y, f, eps, lam)[0]
        assert oc <= ob + 1e-12, (y, f, z, zb)
        # unique minimiser (away from y = 0 where every phase is optimal)
        if abs(y) > 1e-3:
            assert abs(z - zb) < 4 * (R / 800 + R * 2 * math.pi / 720), (y, f, z, zb)


def test_stagm_prox_special_cases():
    lam, eps = 0.7, 0.5
    y = crandn(100)
    f = np.abs(RNG.standard_normal(100))
    # eps -> 0 reduces to the AGM prox (sqrt f + lam |y|)/(1 + lam) sign(y)
    agm = (np.sqrt(f) + lam * np.abs(y)) / (1 + lam) * y / np.abs(y)
    np.testing.assert_allclose(oracle.stagm_prox(y, f, 1e-12, lam), agm, rtol=1e-12)
    # f = 0: prox of |z|^2/2 is lam y / (1 + lam)
    np.testing.assert_allclose(oracle.stagm_prox(y, 0.0, eps, lam), lam * y / (1 + lam), rtol=1e-12)
    # a point on the measured modulus circle is a fixed point of the prox
    yc = np.sqrt(f) * np.exp(1j * RNG.uniform(-3, 3, 100))
    np.testing.assert_allclose(oracle.stagm_prox(yc, f, eps, lam), yc, atol=1e-12)


# ----------------------------------------------------------------------------- operator A
def _dense_A(H, W, w, offs):
    """A as a dense matrix: rows F diag(w) S_j stacked; F built from the DFT definition."""
    m = w.shape[0]
    k = np.arange(m)
    F1 = np.exp(-2j * np.pi * np.outer(k, k) / m) / math.sqrt(m)
    F = np.kron(F1, F1)
    blocks = []
    for r0, c0 in offs:
        S = np.zeros((m * m, H * W))
        for r in range(m):
            for c in range(m):
                S[r * m + c, (r0 + r) * W + (c0 + c)] = 1.0
        blocks.append(F @ np.diag(w.reshape(-1)) @ S)
    return np.vstack(blocks)


def test_forward_adjoint_dense_matrix():
    H, W, m = 9, 8, 4
    offs = np.array([[0, 0], [0, 4], [2, 1], [5, 4], [3, 2]], np.int32)
    w = crandn(m, m)
    u = crandn(H, W)
    A = _dense_A(H, W, w, offs)
    np.testing.assert_allclose(oracle.forward(u, w, offs).reshape(-1), A @ u.reshape(-1), atol=1e-12)
    y = crandn(len(offs), m, m)
    np.testing.assert_allclose(oracle.adjoint(y, w, offs, H, W).reshape(-1),
                               A.conj().T @ y.reshape(-1), atol=1e-12)


def test_adjointness_and_AtA_diagonal():
    """<Au, y> = <u, A^* y>; A^*A = diag(sum_j S_j^T |w|^2) (eq. AtA)."""
    H = W = 40
    m = 16
    offs = synth.raster_offsets(H, m, 6, jitter=2, seed=4)
    w = synth.make_probe(m).astype(np.complex128)
    u = crandn(H, W)
    y = crandn(len(offs), m, m)
    lhs = np.vdot(oracle.forward(u, w, offs).reshape(-1), y.reshape(-1))
    rhs = np.vdot(u.reshape(-1), oracle.adjoint(y, w, offs, H, W).reshape(-1))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    N = np.zeros((H, W))
    for r0, c0 in offs:
        N[r0:r0 + m, c0:c0 + m] += np.abs(w) ** 2
    np.testing.assert_allclose(oracle.adjoint(oracle.forward(u, w, offs), w, offs, H, W), N * u,
                               atol=1e-12)


# ----------------------------------------------------------------------------- geometry
def _width(rect, a, b, axis):
    lo = max(rect[a][axis], rect[b][axis])
    hi = min(rect[a][axis + 2], rect[b][axis + 2])
    return hi - lo


def test_geometry_reproduces_section_4_1():
    g = GOLDEN["e1_two_subdomains"]
    offs = synth.raster_offsets(g["image"], g["probe"], g["step"])
    assert len(offs) == g["n_frames"]
    fs, rect = oracle.geometry(g["image"], g["image"], g["probe"], offs, 1, 2, 0)
    assert np.bincount(fs).tolist() == g["frames_per_subdomain"]
    assert _width(rect, 0, 1, 1) == g["overlap_width"]


@pytest.mark.parametrize("D", GOLDEN["e4_stripes"]["subdomains"])
def test_geometry_reproduces_stripes_of_table_1(D):
    g = GOLDEN["e4_stripes"]
    offs = synth.raster_offsets(g["image"], g["probe"], g["step"])
    assert len(offs) == g["n_frames"]
    fs, rect = oracle.geometry(g["image"], g["image"], g["probe"], offs, 1, D, 0)
    for d in range(D - 1):
        assert _width(rect, d, d + 1, 1) == g["overlap_width"]


@pytest.mark.parametrize("m,step,width", GOLDEN["overlap_rule"]["cases"])
def test_overlap_width_rule(m, step, width):
    n = m + 11 * step
    offs = synth.raster_offsets(n, m, step)
    fs, rect = oracle.geometry(n, n, m, offs, 1, 2, 0)
    assert _width(rect, 0, 1, 1) == width


@pytest.mark.parametrize("grid,ov,jit", [((4, 4), 16, 2), ((3, 5), 0, 0), ((1, 1), 8, 1), ((2, 3), 40, 3)])
def test_geometry_invariants(grid, ov, jit):
    n, m = 300, 32
    offs = synth.raster_offsets(n, m, 12, jitter=jit, seed=9)
    fs, rect = oracle.geometry(n, n, m, offs, grid[0], grid[1], ov)
    # complete frames: every window lies in its subdomain (section 2.1)
    for (r0, c0), d in zip(offs, fs):
        R = rect[d]
        assert R[0] <= r0 and r0 + m <= R[2] and R[1] <= c0 and c0 + m <= R[3]
    # the subdomains cover the image
    cov = np.zeros((n, n), bool)
    for R in rect:
        cov[R[0]:R[2], R[1]:R[3]] = True
    assert cov.all()
    # pair list: symmetric, intersections exact, requested minimum overlap met
    pr, prc = oracle.pairs(rect)
    s = {tuple(p) for p in pr}
    assert all((e, d) in s for d, e in s)
    for (d, e), R in zip(pr, prc):
        assert R[0] == max(rect[d][0], rect[e][0]) and R[3] == min(rect[d][3], rect[e][3])
    for a in range(grid[0]):
        for b in range(grid[1] - 1):
            d = a * grid[1] + b
            assert _width(rect, d, d + 1, 1) >= ov


# ----------------------------------------------------------------------------- ADMM
def _tiny_problem(blind=False, noiseless=True, seed=0, H=14, W=14, m=4, step=2, probe="random"):
    rng = np.random.default_rng(seed)
    offs = synth.raster_offsets(H, m, step, n_cols=W)
    u = (0.5 + 0.5 * rng.random((H, W))) * np.exp(1j * rng.uniform(-1, 1, (H, W)))
    if probe == "random":
        w = (0.5 + rng.random((m, m))) * np.exp(1j * rng.uniform(-2, 2, (m, m)))
    else:
        w = synth.make_probe(m).astype(complex)
    f = np.abs(oracle.forward(u, w, offs)) ** 2
    if not noiseless:
        f = f * (1 + 0.1 * rng.random(f.shape))
    return u, w, offs, f


@pytest.mark.parametrize("grid", [(1, 1), (1, 2), (2, 2), (2, 3)])
def test_noiseless_truth_is_fixed_point(grid):
    """Noiseless truth with zero multipliers satisfies every Step of Algorithm 2."""
    p = synth.small_2sub()
    offs = p.offsets()
    u, w = p.truth().astype(complex), p.probe().astype(complex)
    f = np.abs(oracle.forward(u, w, offs)) ** 2
    a = oracle.ADMM(f, w, offs, 64, 64, grid[0], grid[1], 8, 0.5, 0.1, 0.05, u0=u)
    a.iterate(3)
    np.testing.assert_allclose(a.merge(), u, atol=1e-12)
    assert np.abs(a.get(oracle.GAMMA)).max() < 1e-12
    assert np.abs(a.get(oracle.LAMBDA)).max() < 1e-12 if a.P else True
    assert a.metrics()[0] < 1e-12


def test_blind_noiseless_truth_is_fixed_point():
    """Algorithm 3: (u*, w*) with W_d = w*, zero multipliers, M = I is a fixed point."""
    p = synth.small_2sub()
    offs = p.offsets()
    u, w = p.truth().astype(complex), p.probe().astype(complex)
    f = np.abs(oracle.forward(u, w, offs)) ** 2
    a = oracle.ADMM(f, w, offs, 64, 64, 1, 2, 8, 0.5, 0.1, 0.05, u0=u, blind=True, mu=2.0,
                    gamma=0.3)
    a.iterate(3)
    np.testing.assert_allclose(a.merge(), u, atol=1e-12)
    np.testing.assert_allclose(a.get(oracle.W), w.reshape(-1), atol=1e-12)
    np.testing.assert_allclose(a.get(oracle.WD), np.tile(w.reshape(-1), 2), atol=1e-12)


def _rect_index(rect, d, R, C):
    r0, c0, r1, c1 = rect[d]
    return (R - r0) * (c1 - c0) + (C - c0)


def _scramble_state(a, rng, blind=False):
    """Random multipliers and iterates: the subproblem pins must hold from any state."""
    for k in (oracle.U, oracle.GAMMA, oracle.LAMBDA) + ((oracle.WD, oracle.DELTA) if blind else ()):
        n = len(a.get(k))
        if n:
            a.set(k, 0.3 * crandn(n, rng=rng) + (1.0 if k in (oracle.U, oracle.WD) else 0.0))


@pytest.mark.parametrize("grid", [(1, 1), (1, 2), (2, 2)])
def test_step3_u_is_least_squares_minimiser(grid):
    """Step 3 of Algorithm 2 against a dense least-squares solve of its subproblem
    min_u eta/2 ||A_d u + Gamma^{n+1} - z^{n+1}||^2 + r/2 sum_e ||pi u - v^{n+1} + Lambda^n||^2."""
    H = W = 14
    m = 4
    u, w, offs, f = _tiny_problem(noiseless=False, seed=1)
    eta, r, eps = 0.3, 0.7, 0.5
    a = oracle.ADMM(f, w, offs, H, W, grid[0], grid[1], 2, eps, eta, r)
    rng = np.random.default_rng(7)
    _scramble_state(a, rng)
    lam_n = a.get(oracle.LAMBDA)
    fs, rect = oracle.geometry(H, W, m, offs, grid[0], grid[1], 2)
    pr, prc = oracle.pairs(rect)
    a.iterate(1)
    z, gam, v, un = a.get(oracle.Z), a.get(oracle.GAMMA), a.get(oracle.V), a.get(oracle.U)
    lam_off = np.concatenate([[0], np.cumsum([(R[2] - R[0]) * (R[3] - R[1]) for R in prc])]).astype(int)
    u_off = np.concatenate([[0], np.cumsum([(R[2] - R[0]) * (R[3] - R[1]) for R in rect])]).astype(int)
    mm = m * m
    for d in range(len(rect)):
        r0, c0, r1, c1 = rect[d]
        hd, wd = r1 - r0, c1 - c0
        js = np.where(fs == d)[0]
        loc = offs[js] - np.array([r0, c0])
        rows, rhs = [], []
        if len(js):
            Ad = _dense_A(hd, wd, w, loc)
            rows.append(math.sqrt(eta) * Ad)
            rhs.append(math.sqrt(eta) * (z.reshape(-1, mm)[js] - gam.reshape(-1, mm)[js]).reshape(-1))
        for k, (dd, e) in enumerate(pr):
            if dd != d:
                continue
            R = prc[k]
            for RR in range(R[0], R[2]):
                for CC in range(R[1], R[3]):
                    row = np.zeros(hd * wd)
                    row[_rect_index(rect, d, RR, CC)] = math.sqrt(r)
                    i = lam_off[k] + (RR - R[0]) * (R[3] - R[1]) + (CC - R[1])
                    rows.append(row[None, :])
                    rhs.append(np.array([math.sqrt(r) * (v[i] - lam_n[i])]))
        M = np.vstack(rows)
        b = np.concatenate(rhs)
        sol = np.linalg.lstsq(M, b, rcond=None)[0]
        np.testing.assert_allclose(un[u_off[d]:u_off[d + 1]], sol, atol=1e-10)


def test_one_subdomain_is_the_whole_domain_iteration():
    """With one subdomain there are no overlap pairs: the consensus penalty r drops
    out (iterates identical for any r) and one iteration is the ADMM of the
    undecomposed problem -- z = Prox(Gamma + A u), Gamma += A u - z,
    u = A^*(z - Gamma) / diag(A^* A) -- written with the oracle's operators."""
    H = W = 14
    m = 4
    u, w, offs, f = _tiny_problem(noiseless=False, seed=2)
    eta, eps = 0.4, 0.5
    runs = []
    for r in (0.05, 4e3):
        a = oracle.ADMM(f, w, offs, H, W, 1, 1, 0, eps, eta, r)
        a.iterate(3)
        runs.append([a.get(k) for k in (oracle.U, oracle.GAMMA)])
    for x, y in zip(*runs):
        assert np.array_equal(x, y)
    a = oracle.ADMM(f, w, offs, H, W, 1, 1, 0, eps, eta, 1.0)
    a.iterate(2)
    u_n, g_n = a.get(oracle.U).reshape(H, W), a.get(oracle.GAMMA).reshape(-1, m, m)
    a.iterate(1)
    Au = oracle.forward(u_n, w, offs)
    y = g_n + Au
    z = oracle.stagm_prox(y.reshape(-1), f.reshape(-1), eps, eta).reshape(y.shape)
    g1 = y - z
    illum = np.zeros((H, W))
    for r0, c0 in offs:
        illum[r0:r0 + m, c0:c0 + m] += np.abs(w) ** 2
    u1 = oracle.adjoint(z - g1, w, offs, H, W) / illum
    np.testing.assert_allclose(a.get(oracle.GAMMA).reshape(g1.shape), g1, atol=1e-12)
    np.testing.assert_allclose(a.get(oracle.U).reshape(H, W), u1, atol=1e-10)


def test_step1_step2_optimality_conditions():
    """eq. (Stationary1): grad G(z^{n+1}) = eta Gamma^{n+1} and v^{n+1} averages pi u^n + Lambda^n;
    eq. (updateM-2): Lambda^{n+1} = Lambda^n + pi u^{n+1} - v^{n+1}."""
    H = W = 14
    m = 4
    u, w, offs, f = _tiny_problem(noiseless=False, seed=2)
    eta, r, eps = 0.4, 0.9, 0.5
    a = oracle.ADMM(f, w, offs, H, W, 2, 2, 2, eps, eta, r)
    _scramble_state(a, np.random.default_rng(3))
    u_n, lam_n = a.get(oracle.U), a.get(oracle.LAMBDA)
    a.iterate(1)
    z, gam = a.get(oracle.Z), a.get(oracle.GAMMA)
    np.testing.assert_allclose(oracle.stagm_grad(z, f.reshape(-1), eps), eta * gam, atol=1e-11)
    fs, rect = oracle.geometry(H, W, m, offs, 2, 2, 2)
    pr, prc = oracle.pairs(rect)
    v, lam1, u1 = a.get(oracle.V), a.get(oracle.LAMBDA), a.get(oracle.U)
    u_off = np.concatenate([[0], np.cumsum([(R[2] - R[0]) * (R[3] - R[1]) for R in rect])]).astype(int)
    lam_off = np.concatenate([[0], np.cumsum([(R[2] - R[0]) * (R[3] - R[1]) for R in prc])]).astype(int)
    idx = {tuple(p): k for k, p in enumerate(pr)}
    for k, (d, e) in enumerate(pr):
        R = prc[k]
        for RR in range(R[0], R[2]):
            for CC in range(R[1], R[3]):
                o = (RR - R[0]) * (R[3] - R[1]) + (CC - R[1])
                i_de, i_ed = lam_off[k] + o, lam_off[idx[(e, d)]] + o
                ud = u_n[u_off[d] + _rect_index(rect, d, RR, CC)]
                ue = u_n[u_off[e] + _rect_index(rect, e, RR, CC)]
                # gradient of r/2 (|v - pi u_d - Lambda_de|^2 + |v - pi u_e - Lambda_ed|^2) vanishes
                assert abs((v[i_de] - ud - lam_n[i_de]) + (v[i_de] - ue - lam_n[i_ed])) < 1e-12
                assert abs(v[i_de] - v[i_ed]) < 1e-15
                ud1 = u1[u_off[d] + _rect_index(rect, d, RR, CC)]
                assert abs(lam1[i_de] - (lam_n[i_de] + ud1 - v[i_de])) < 1e-12


def _aug_lagrangian(a, f, w, offs, H, W, m, grid, eps, eta, r, fs, rect, pr, prc):
    """eq. (augLag-multi-Domain) evaluated from the oracle state with numpy's FFT."""
    u, z, gam, lam, v = (a.get(k) for k in (oracle.U, oracle.Z, oracle.GAMMA, oracle.LAMBDA, oracle.V))
    mm = m * m
    u_off = np.concatenate([[0], np.cumsum([(R[2] - R[0]) * (R[3] - R[1]) for R in rect])]).astype(int)
    Lval = np.sum(oracle.stagm_g(z, f.reshape(-1), eps))
    for j, (r0, c0) in enumerate(offs):
        d = fs[j]
        R = rect[d]
        ud = u[u_off[d]:u_off[d + 1]].reshape(R[2] - R[0], R[3] - R[1])
        Au = np.fft.fft2(w * ud[r0 - R[0]:r0 - R[0] + m, c0 - R[1]:c0 - R[1] + m], norm="ortho").reshape(-1)
        res = Au - z[j * mm:(j + 1) * mm]
        Lval += eta * (np.real(np.vdot(gam[j * mm:(j + 1) * mm], res)) + 0.5 * np.vdot(res, res).real)
    lam_off = np.concatenate([[0], np.cumsum([(R[2] - R[0]) * (R[3] - R[1]) for R in prc])]).astype(int)
    for k, (d, e) in enumerate(pr):
        R = prc[k]
        Rd = rect[d]
        ud = u[u_off[d]:u_off[d + 1]].reshape(Rd[2] - Rd[0], Rd[3] - Rd[1])
        pu = ud[R[0] - Rd[0]:R[2] - Rd[0], R[1] - Rd[1]:R[3] - Rd[1]].reshape(-1)
        res = pu - v[lam_off[k]:lam_off[k + 1]]
        Lval += r * (np.real(np.vdot(lam[lam_off[k]:lam_off[k + 1]], res)) + 0.5 * np.vdot(res, res).real)
    return Lval


def test_augmented_lagrangian_nonincreasing_in_K():
    """Lemma 2.4 / Theorem 3.1: for (r, eta) in the set K the augmented Lagrangian does not increase."""
    H = W = 14
    m = 4
    u, w, offs, f = _tiny_problem(noiseless=False, seed=5)
    eps = 0.5
    L = 2 / eps - 1
    eta = 8 * L + 2 * L * L + 20  # comfortably inside K (eq. paramsSet_multi)
    grid = (1, 2)
    fs, rect = oracle.geometry(H, W, m, offs, *grid, 2)
    pr, prc = oracle.pairs(rect)
    N = np.zeros((H, W))
    for r0, c0 in offs:
        N[r0:r0 + m, c0:c0 + m] += np.abs(w) ** 2
    r = 4 * eta * N.max() ** 2 + 10
    a = oracle.ADMM(f, w, offs, H, W, *grid, 2, eps, eta, r)
    a.iterate(1)
    vals = []
    for _ in range(25):
        a.iterate(1)
        vals.append(_aug_lagrangian(a, f, w, offs, H, W, m, grid, eps, eta, r, fs, rect, pr, prc))
    vals = np.array(vals)
    assert np.all(np.diff(vals) <= 1e-9 * np.abs(vals[:-1]).max()), vals


@pytest.mark.parametrize("grid,ov", [((1, 2), 2), ((2, 2), 2)])
def test_operator_norms_are_spectral_norms(grid, ov):
    """Lemma 2.4's ||A_d^* A_d|| and ||pi_{d,e} A_d^*||^2 equal the largest
    squared singular values of the dense operators (F diag(w) S_j restricted to
    Omega_d; its adjoint restricted to the overlap rows)."""
    H = W = 14
    m = 4
    u, w, offs, f = _tiny_problem(seed=7, H=H, W=W)
    fs, rect = oracle.geometry(H, W, m, offs, *grid, ov)
    pr, prc = oracle.pairs(rect)
    a_want, b_want = 0.0, 0.0
    for d, R in enumerate(rect):
        cols = np.array([r * W + c for r in range(R[0], R[2]) for c in range(R[1], R[3])])
        Ad = _dense_A(H, W, w, offs[fs == d])[:, cols]
        a_want = max(a_want, np.linalg.norm(Ad, 2) ** 2)
        for (d0, _e), P in zip(pr, prc):
            if d0 != d:
                continue
            rows = [i for i, px in enumerate(cols) if P[0] <= px // W < P[2] and P[1] <= px % W < P[3]]
            b_want = max(b_want, np.linalg.norm(Ad.conj().T[rows, :], 2) ** 2)
    a, b = oracle.operator_norms(w, offs, H, W, *grid, ov)
    assert len(pr) > 0
    assert abs(a - a_want) < 1e-9 * a_want and abs(b - b_want) < 1e-9 * b_want, (a, a_want, b, b_want)


def test_params_in_K_lie_in_K():
    """The sufficient choice after eq. (paramsSet) satisfies its three
    inequalities; parameters below the bounds fail them."""
    from paper_2011_00162_gb300 import adaptive
    for norms in [(16.0, 9.0), (1.0, 0.25), (300.0, 300.0), (2.0, 0.0)]:
        for eps in (0.2, 0.5, 0.9):
            r, eta = adaptive.params_in_K(norms, eps)
            assert adaptive.in_K(r, eta, norms, eps), (norms, eps, r, eta)
            L = 2 / eps - 1
            assert eta > 6 * L + 2 * L * L and r > 2 * norms[0] * eta
            assert not adaptive.in_K(r, 0.5, norms, eps)                 # eta < 1
            assert not adaptive.in_K(eta * 2 * norms[0], eta, norms, eps)  # r = c0 eta (not >)
            assert not adaptive.in_K(r, 3 * L, norms, eps)               # (eta - 3L)/2 - ... < 0
    with pytest.raises(ValueError):
        adaptive.params_in_K((1.0, 1.0), 0.5, margin=1.0)


def test_augmented_lagrangian_nonincreasing_for_selected_params():
    """Lemma 2.4 with (r, eta) chosen from the measured operator norms."""
    from paper_2011_00162_gb300 import adaptive
    H = W = 14
    m = 4
    u, w, offs, f = _tiny_problem(noiseless=False, seed=8)
    eps, grid = 0.5, (1, 2)
    r, eta = adaptive.params_in_K(oracle.operator_norms(w, offs, H, W, *grid, 2), eps)
    fs, rect = oracle.geometry(H, W, m, offs, *grid, 2)
    pr, prc = oracle.pairs(rect)
    a = oracle.ADMM(f, w, offs, H, W, *grid, 2, eps, eta, r)
    a.iterate(1)
    vals = []
    for _ in range(25):
        a.iterate(1)
        vals.append(_aug_lagrangian(a, f, w, offs, H, W, m, grid, eps, eta, r, fs, rect, pr, prc))
    vals = np.array(vals)
    assert np.all(np.diff(vals) <= 1e-9 * np.abs(vals[:-1]).max()), vals


def test_blind_W_and_U_are_least_squares_minimisers():
    """Algorithm 3, eqs. (blind_W) and (blind_U), against dense least-squares solves."""
    H = W = 12
    m = 4
    u, w, offs, f = _tiny_problem(noiseless=False, seed=6, H=H, W=W)
    eta, r, eps, mu, gamma = 0.3, 0.6, 0.5, 0.8, 0.25
    grid = (1, 2)
    a = oracle.ADMM(f, w, offs, H, W, *grid, 2, eps, eta, r, blind=True, mu=mu, gamma=gamma)
    _scramble_state(a, np.random.default_rng(11), blind=True)
    u_n, Wd_n, Dl_n, lam_n = (a.get(k) for k in (oracle.U, oracle.WD, oracle.DELTA, oracle.LAMBDA))
    a.iterate(1)
    z, gam, v, w1, Wd1, u1, Dl1 = (a.get(k) for k in (oracle.Z, oracle.GAMMA, oracle.V, oracle.W,
                                                      oracle.WD, oracle.U, oracle.DELTA))
    D = 2
    mm = m * m
    # w-update: minimiser of mu/2 sum_d ||Delta_d + W_d - w||^2 with M = I
    np.testing.assert_allclose(w1, (Dl_n + Wd_n).reshape(D, mm).mean(0), atol=1e-12)
    fs, rect = oracle.geometry(H, W, m, offs, *grid, 2)
    pr, prc = oracle.pairs(rect)
    u_off = np.concatenate([[0], np.cumsum([(R[2] - R[0]) * (R[3] - R[1]) for R in rect])]).astype(int)
    lam_off = np.concatenate([[0], np.cumsum([(R[2] - R[0]) * (R[3] - R[1]) for R in prc])]).astype(int)
    k1 = np.arange(m)
    F1 = np.exp(-2j * np.pi * np.outer(k1, k1) / m) / math.sqrt(m)
    F = np.kron(F1, F1)
    for d in range(D):
        R = rect[d]
        hd, wd = R[2] - R[0], R[3] - R[1]
        ud_n = u_n[u_off[d]:u_off[d + 1]].reshape(hd, wd)
        js = np.where(fs == d)[0]
        # W-subproblem: min eta/2 sum_j ||F(W o S_j u^n) - z_j + Gamma_j||^2 + mu/2 ||W - w + Delta||^2
        rows = [math.sqrt(eta) * F @ np.diag(ud_n[o[0] - R[0]:o[0] - R[0] + m, o[1] - R[1]:o[1] - R[1] + m].reshape(-1))
                for o in offs[js]]
        rows.append(math.sqrt(mu) * np.eye(mm))
        rhs = [math.sqrt(eta) * (z.reshape(-1, mm)[j] - gam.reshape(-1, mm)[j]) for j in js]
        rhs.append(math.sqrt(mu) * (w1 - Dl_n.reshape(D, mm)[d]))
        solW = np.linalg.lstsq(np.vstack(rows), np.concatenate(rhs), rcond=None)[0]
        np.testing.assert_allclose(Wd1.reshape(D, mm)[d], solW, atol=1e-10)
        # U-subproblem with W^{n+1} and the proximal term gamma/2 ||U - U^n||^2
        Wn1 = Wd1.reshape(D, mm)[d].reshape(m, m)
        rows = [math.sqrt(eta) * _dense_A(hd, wd, Wn1, offs[js] - np.array([R[0], R[1]]))]
        rhs = [math.sqrt(eta) * (z.reshape(-1, mm)[js] - gam.reshape(-1, mm)[js]).reshape(-1)]
        for k, (dd, e) in enumerate(pr):
            if dd != d:
                continue
            P = prc[k]
            for RR in range(P[0], P[2]):
                for CC in range(P[1], P[3]):
                    row = np.zeros(hd * wd)
                    row[_rect_index(rect, d, RR, CC)] = math.sqrt(r)
                    i = lam_off[k] + (RR - P[0]) * (P[3] - P[1]) + (CC - P[1])
                    rows.append(row[None, :])
                    rhs.append(np.array([math.sqrt(r) * (v[i] - lam_n[i])]))
        rows.append(math.sqrt(gamma) * np.eye(hd * wd))
        rhs.append(math.sqrt(gamma) * ud_n.reshape(-1))
        solU = np.linalg.lstsq(np.vstack(rows), np.concatenate(rhs), rcond=None)[0]
        np.testing.assert_allclose(u1[u_off[d]:u_off[d + 1]], solU, atol=1e-10)
        # eq. admm_Delta
        np.testing.assert_allclose(Dl1.reshape(D, mm)[d], Dl_n.reshape(D, mm)[d] + Wd1.reshape(D, mm)[d] - w1,
                                   atol=1e-12)


def test_blind_fourier_mask_projects_probe():
    """eq. (blind_w) with a support mask: F w^{n+1} vanishes off the support."""
    H = W = 12
    m = 4
    u, w, offs, f = _tiny_problem(noiseless=False, seed=8, H=H, W=W)
    mask = np.ones((m, m))
    mask[1:3, :] = 0
    a = oracle.ADMM(f, w, offs, H, W, 1, 2, 2, 0.5, 0.3, 0.6, blind=True, mu=0.8, mask=mask)
    a.iterate(2)
    Fw = np.fft.fft2(a.get(oracle.W).reshape(m, m), norm="ortho")
    assert np.abs(Fw[mask == 0]).max() < 1e-13
    assert np.abs(Fw[mask == 1]).max() > 1e-3


def test_merge_averages_overlaps():
    p = synth.small_2sub()
    offs = p.offsets()
    u, w = p.truth().astype(complex), p.probe().astype(complex)
    f = np.abs(oracle.forward(u, w, offs)) ** 2
    a = oracle.ADMM(f, w, offs, 64, 64, 2, 2, 8, 0.5, 0.1, 0.05, u0=u)
    np.testing.assert_allclose(a.merge(), u, atol=0)
    uu = a.get(oracle.U)
    a.set(oracle.U, uu * 0 + 2.0)
    np.testing.assert_allclose(a.merge(), 2.0)


def test_noiseless_reconstruction_converges():
    """From u = 1 the nonblind iteration drives RF down on noiseless data (section 4.1)."""
    p = synth.small_2sub()
    offs = p.offsets()
    u, w = p.truth(), p.probe()
    f = (np.abs(oracle.forward(u, w, offs)) ** 2).astype(np.float32)
    a = oracle.ADMM(f, w, offs, 64, 64, 1, 2, 8, p.eps, p.eta, p.r)
    a.iterate(1)
    rf1 = a.metrics()[0]
    a.iterate(49)
    assert a.metrics()[0] < 0.1 * rf1


# ----------------------------------------------------------------------------- loss and gradient
def test_loss_gradient_finite_differences():
    H = W = 12
    m = 4
    u, w, offs, f = _tiny_problem(noiseless=False, seed=9, H=H, W=W)
    rng = np.random.default_rng(10)
    u = u * (1 + 0.3 * crandn(H, W, rng=rng))
    w = w * (1 + 0.3 * crandn(m, m, rng=rng))
    eps = 0.5
    L0, gu, gw = oracle.loss_grad(u, w, offs, f, eps)
    h = 1e-6
    for _ in range(12):
        i, k = rng.integers(0, H), rng.integers(0, W)
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            up, um = u.copy(), u.copy()
            up[i, k] += h * unit
            um[i, k] -= h * unit
            fd = (oracle.loss_grad(up, w, offs, f, eps)[0] - oracle.loss_grad(um, w, offs, f, eps)[0]) / (2 * h)
            assert abs(fd - part(gu[i, k])) < 1e-6 * max(1.0, abs(fd))
        i, k = rng.integers(0, m), rng.integers(0, m)
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            wp, wm = w.copy(), w.copy()
            wp[i, k] += h * unit
            wm[i, k] -= h * unit
            fd = (oracle.loss_grad(u, wp, offs, f, eps)[0] - oracle.loss_grad(u, wm, offs, f, eps)[0]) / (2 * h)
            assert abs(fd - part(gw[i, k])) < 1e-6 * max(1.0, abs(fd))


def test_loss_reduces_to_agm_and_vanishes_at_truth():
    H = W = 20
    m = 8
    u, w, offs, f = _tiny_problem(noiseless=True, seed=12, H=H, W=W, m=m, step=3)
    L, gu, gw = oracle.loss_grad(u, w, offs, f, 0.5)
    assert abs(L) < 1e-20 and np.abs(gu).max() < 1e-12 and np.abs(gw).max() < 1e-12
    u2 = u * np.exp(1j * 0.3 * np.random.default_rng(1).standard_normal((H, W)))
    L2 = oracle.loss_grad(u2, w, offs, f, 1e-12)[0]
    frames = np.stack([np.fft.fft2(w * u2[r:r + m, c:c + m], norm="ortho") for r, c in offs])
    agm = 0.5 * np.sum((np.abs(frames) - np.sqrt(f)) ** 2)
    assert abs(L2 - agm) < 1e-10 * agm


# ----------------------------------------------------------------------------- data-driven initial probe
@pytest.mark.parametrize("m", [16, 64])
def test_probe_init_recovers_a_probe_with_positive_spectrum(m):
    """Section 4.2's w0 = (1/J) sum_j F^* sqrt(f_j): when every frame measures
    |F w|^2 of a probe whose spectrum F w = a is real and positive, sqrt(f_j) = a
    and the mean of F^* a over the frames is w itself (numpy builds w)."""
    rng = np.random.default_rng(m)
    a = 0.1 + rng.random((m, m))
    w = np.fft.ifft2(a, norm="ortho")
    f = np.repeat((a * a)[None], 5, axis=0)
    assert np.abs(oracle.probe_init(f) - w).max() < 1e-12 * np.abs(w).max()


def test_probe_init_is_the_mean_over_frames_and_unitary():
    rng = np.random.default_rng(2)
    m = 32
    amps = [rng.random((m, m)) for _ in range(3)]
    f = np.stack([x * x for x in amps])
    expect = sum(np.fft.ifft2(x, norm="ortho") for x in amps) / 3.0
    assert np.abs(oracle.probe_init(f) - expect).max() < 1e-13
    # one bright zero frequency c^2: F^* gives the constant c / m everywhere
    g = np.zeros((1, m, m))
    g[0, 0, 0] = 9.0
    assert np.abs(oracle.probe_init(g) - 3.0 / m).max() < 1e-15


@pytest.mark.parametrize("m,n,step", [(12, 48, 4), (6, 30, 3)])
def test_non_power_of_two_probe_fixed_point_and_dense_operator(m, n, step):
    """Probe sides that are not powers of two: the forward operator equals the
    dense matrix F diag(w) S_j, and the noiseless truth stays a fixed point."""
    offs = synth.raster_offsets(n, m, step, jitter=1, seed=2)
    w = synth.make_probe(m).astype(np.complex128)
    u = synth.make_truth(n, m, offs, 3).astype(np.complex128)
    if n * n <= 900:
        A = _dense_A(n, n, w, offs)
        np.testing.assert_allclose(oracle.forward(u, w, offs).reshape(-1), A @ u.reshape(-1), atol=1e-12)
    f = np.abs(oracle.forward(u, w, offs)) ** 2
    a = oracle.ADMM(f, w, offs, n, n, 2, 2, 4, 0.5, 0.5, 0.2, u0=u)
    a.iterate(3)
    np.testing.assert_allclose(a.merge(), u, atol=1e-11)
    assert np.abs(a.get(oracle.GAMMA)).max() < 1e-11


# ----------------------------------------------------------------------------- penalty changes
def _noisy_small():
    p = synth.Problem("pc", 96, 16, 4, 1, 2, 2, 8, 1e4, 1, eta=2.0, r=0.5, seed=6)
    offs = p.offsets()
    u, w = p.truth(), p.probe()
    f = synth.poissonize(np.abs(oracle.forward(u, w, offs)) ** 2, p.peak, 3)
    return p, offs, w, f


def test_penalty_change_keeps_unscaled_multipliers():
    """Changing (eta, r) rescales the scaled multipliers so that eta*Gamma and
    r*Lambda stay (Boyd et al. 2011, 3.4.1).  The unscaled multipliers of a run
    that has nearly settled do not depend on the penalties, so with the
    rescaling the next step moves about as far as a step with unchanged
    penalties; left unscaled, the same change makes the run jump."""
    p, offs, w, f = _noisy_small()
    a = oracle.ADMM(f, w, offs, p.n, p.n, 2, 2, 8, 0.5, 2.0, 0.5)
    a.iterate(400)
    g0, l0, u0 = a.get(oracle.GAMMA), a.get(oracle.LAMBDA), a.get(oracle.U)
    a.set_penalties(2.0, 0.5)  # same values: nothing changes
    assert np.array_equal(a.get(oracle.GAMMA), g0) and np.array_equal(a.get(oracle.LAMBDA), l0)

    def step(eta, r, rescale):
        b = oracle.ADMM(f, w, offs, p.n, p.n, 2, 2, 8, 0.5, 2.0 if rescale else eta, 0.5 if rescale else r)
        for k, v in ((oracle.U, u0), (oracle.GAMMA, g0), (oracle.LAMBDA, l0)):
            b.set(k, v)
        if rescale:
            b.set_penalties(eta, r)
            np.testing.assert_allclose(eta * b.get(oracle.GAMMA), 2.0 * g0, rtol=1e-14, atol=1e-15)
            np.testing.assert_allclose(r * b.get(oracle.LAMBDA), 0.5 * l0, rtol=1e-14, atol=1e-15)
        b.iterate(1)
        return np.linalg.norm(b.get(oracle.U) - u0) / np.linalg.norm(u0)

    base = step(2.0, 0.5, True)
    for eta, r in [(4.0, 2.0), (2.0, 2.0), (8.0, 0.5)]:
        kept, jumped = step(eta, r, True), step(eta, r, False)
        assert kept < 2 * base and jumped > 5 * kept, (eta, r, base, kept, jumped)


def test_consensus_residual():
    """0 for one subdomain and at the noiseless truth; a constant c added to one
    subdomain's copy gives |c| sqrt(2 * overlap pixels of its pairs) / ||u||."""
    p = synth.small_2sub()
    offs = p.offsets()
    u, w = p.truth().astype(complex), p.probe().astype(complex)
    f = np.abs(oracle.forward(u, w, offs)) ** 2
    one = oracle.ADMM(f, w, offs, 64, 64, 1, 1, 0, 0.5, 0.1, 0.05, u0=u)
    assert one.consensus() == 0.0
    a = oracle.ADMM(f, w, offs, 64, 64, 2, 2, 8, 0.5, 0.1, 0.05, u0=u)
    assert a.consensus() < 1e-15
    fs, rect = oracle.geometry(64, 64, 16, offs, 2, 2, 8)
    pr, prc = oracle.pairs(rect)
    sizes = [(r[2] - r[0]) * (r[3] - r[1]) for r in rect]
    uu = a.get(oracle.U).copy()
    c = 0.25 - 0.5j
    uu[:sizes[0]] += c
    a.set(oracle.U, uu)
    ov = sum((q[2] - q[0]) * (q[3] - q[1]) for (d, e), q in zip(pr, prc) if d == 0)
    expect = abs(c) * np.sqrt(2 * ov) / np.linalg.norm(uu)
    assert abs(a.consensus() - expect) < 1e-12 * expect


def test_snr_definition():
    """Section 4's SNR of a recovery u_r against the truth u_g, normalised by
    ||u_r||^2 as printed: a 10% scaling of the truth gives 20 dB plus the norm
    ratio, a global phase of the recovery does not count, and a perturbation of
    known energy gives its ratio."""
    ug = crandn(40, 40)
    assert abs(oracle.snr(1.1 * ug, ug) - (20.0 + 10 * np.log10(1.21))) < 1e-9
    assert abs(oracle.snr(0.9 * ug * np.exp(1.3j), ug) - (20.0 + 10 * np.log10(0.81))) < 1e-9
    d = crandn(40, 40)
    d -= np.vdot(ug, d) / np.vdot(ug, ug) * ug   # orthogonal to ug: no phase to remove
    d *= 0.01 * np.linalg.norm(ug) / np.linalg.norm(d)
    assert abs(oracle.snr(ug + d, ug) - (40.0 + 10 * np.log10(1.0001))) < 1e-6


# ----------------------------------------------------------------------------- RF and RE
def _metrics_case(blind):
    """A noisy 2 x 2 problem run a few iterations, so that RF, RE and the
    multipliers are all away from their trivial values."""
    p = synth.Problem("rfre", 96, 16, 6, 1, 2, 2, 8, 1e3, 1, eta=2.0, r=0.5, seed=9)
    offs = p.offsets()
    u, w = p.truth(), p.probe()
    f = synth.poissonize(np.abs(oracle.forward(u, w, offs)) ** 2, p.peak, 4).astype(np.float64)
    w0 = w if not blind else synth.gaussian_probe(p.m)
    a = oracle.ADMM(f, w0, offs, p.n, p.n, 2, 2, 8, 0.5, 2.0, 0.5, blind=blind, mu=1.0,
                    gamma=0.1 if blind else 0.0)
    a.iterate(3)
    fs, rect = oracle.geometry(p.n, p.n, p.m, offs, 2, 2, 8)
    return a, f, offs, fs, rect, p.m


def _split_u(u, rect):
    out, k = [], 0
    for r0, c0, r1, c1 in rect:
        n = (r1 - r0) * (c1 - c0)
        out.append(u[k:k + n].reshape(r1 - r0, c1 - c0))
        k += n
    return out


def _rf_numpy(ud, Wd, f, offs, fs, rect, m, norm="sqrt"):
    """Section 4's RF written with numpy: sum_j || |F(W o S_j u_d)| - sqrt f_j ||_1
    over sum_j || sqrt f_j ||_1 (norm="sqrt"); norm="f" is the wrong normaliser."""
    num = 0.0
    for j, (r0, c0) in enumerate(offs):
        d = fs[j]
        R0, C0 = rect[d][0], rect[d][1]
        psi = Wd[d] * ud[d][r0 - R0:r0 - R0 + m, c0 - C0:c0 - C0 + m]
        num += np.abs(np.abs(np.fft.fft2(psi, norm="ortho")) - np.sqrt(f[j])).sum()
    return num / (np.sqrt(f).sum() if norm == "sqrt" else f.sum())


def _re_numpy(u_old, u_new, by="new"):
    """RE = max_d ||u_d^{n+1} - u_d^n|| / ||u_d^{n+1}|| (by="old" is the wrong norm)."""
    return max(np.linalg.norm(b - a) / np.linalg.norm(b if by == "new" else a)
               for a, b in zip(u_old, u_new))


@pytest.mark.parametrize("blind", [False, True])
def test_rf_re_match_their_definitions(blind):
    """The oracle's RF (of the iterate entering the iteration, blind: with the
    subdomain probes W_d^n of Step 1) and RE (relative to u^{n+1}) of section 4,
    recomputed with numpy from the state captured around one iteration.  The
    plausible misreadings -- Sigma f as the normaliser, RF of u^{n+1}, RE against
    ||u^n|| -- differ from both by far more than the tolerance."""
    a, f, offs, fs, rect, m = _metrics_case(blind)
    D = len(rect)
    u_old = _split_u(a.get(oracle.U).copy(), rect)
    Wd = (a.get(oracle.WD).reshape(D, m, m).copy() if blind
          else np.broadcast_to(a.get(oracle.W).reshape(m, m), (D, m, m)))
    a.iterate(1)
    rf, re = a.metrics()
    u_new = _split_u(a.get(oracle.U).copy(), rect)
    rf_np = _rf_numpy(u_old, Wd, f, offs, fs, rect, m)
    re_np = _re_numpy(u_old, u_new)
    assert abs(rf - rf_np) <= 1e-12 * rf_np, (rf, rf_np)
    assert abs(re - re_np) <= 1e-12 * re_np, (re, re_np)
    # the misreadings are told apart
    wrong = {
        "sum f normaliser": _rf_numpy(u_old, Wd, f, offs, fs, rect, m, norm="f"),
        "RF of u^{n+1}": _rf_numpy(u_new, Wd if not blind else a.get(oracle.WD).reshape(D, m, m),
                                   f, offs, fs, rect, m),
    }
    for name, v in wrong.items():
        assert abs(v - rf) > 1e-6 * rf, name
    assert abs(_re_numpy(u_old, u_new, by="old") - re) > 1e-6 * re
    assert rf > 1e-3 and re > 1e-4
