"""Seeded synthetic inputs standing in for the paper's test sample and probe.

The paper's experiments (section 4) use a complex sample built from two real
images (amplitude and phase), a 64 x 64 zone-plate probe, raster scans, and
Poisson-noisy intensities; none of those images ships with the paper.  This
module generates inputs of the same roles, shapes and value ranges from a
seed.  It contains none of the reconstruction method's arithmetic: it makes
the sample, the probe, the scan positions and the noise, and both the CUDA
path and the CPU oracle consume exactly these arrays.  The noiseless
intensities |F(w o S_j u)|^2 are *not* made here (they are the forward model);
callers compute them with the oracle (tests) or the library's forward
operator (benchmark) and then call :func:`poissonize`.

Recipe (all arrays FP32-representable so both sides start from equal values):

* sample: two white-noise fields, Gaussian-blurred (sigma = N/16, periodic),
  min/max mapped to amplitude [0.5, 1] and phase [-pi/2, pi/2]; pixels that no
  probe disk reaches are set to 1 (the paper's samples sit in vacuum with a
  boundary of ones, section 4);
* probe: a disk of radius R (default 0.375 m) apodised by a Gaussian of
  sigma = R/2, with quadratic phase exp(i pi rho^2 / R^2), scaled to max |w| = 1;
* scan: raster grid with `step`; interior positions get seeded uniform integer
  jitter in [-jitter, jitter] per axis, clamped to the image; the first and
  last position of each axis are not jittered in that axis;
* noise: f = Poisson(kappa f_clean) / kappa with kappa = peak / max(f_clean).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def _minmax(x: np.ndarray) -> np.ndarray:
    lo, hi = float(x.min()), float(x.max())
    return (x - lo) / (hi - lo) if hi > lo else np.zeros_like(x)


def smooth_field(n: int, rng: np.random.Generator, sigma: float) -> np.ndarray:
    """White Gaussian noise blurred with a periodic Gaussian kernel of width sigma."""
    white = rng.standard_normal((n, n))
    k = np.fft.fftfreq(n)
    g = np.exp(-2.0 * (math.pi * sigma) ** 2 * (k[:, None] ** 2 + k[None, :] ** 2))
    return np.real(np.fft.ifft2(np.fft.fft2(white) * g))


def make_image(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    amp = 0.5 + 0.5 * _minmax(smooth_field(n, rng, n / 16.0))
    phase = -0.5 * math.pi + math.pi * _minmax(smooth_field(n, rng, n / 16.0))
    return (amp * np.exp(1j * phase)).astype(np.complex64)


def probe_radius(m: int) -> float:
    return 0.375 * m


def make_probe(m: int, radius: float | None = None) -> np.ndarray:
    R = probe_radius(m) if radius is None else float(radius)
    c = 0.5 * (m - 1)
    yy, xx = np.mgrid[0:m, 0:m].astype(np.float64)
    rho2 = (yy - c) ** 2 + (xx - c) ** 2
    amp = np.exp(-rho2 / (2.0 * (R / 2.0) ** 2)) * (rho2 <= R * R)
    w = amp * np.exp(1j * math.pi * rho2 / (R * R))
    w /= np.abs(w).max()
    return w.astype(np.complex64)


def gaussian_probe(m: int, sigma: float | None = None) -> np.ndarray:
    """Initial guess for blind runs: a real Gaussian of width m/8, max 1."""
    s = m / 8.0 if sigma is None else float(sigma)
    c = 0.5 * (m - 1)
    yy, xx = np.mgrid[0:m, 0:m].astype(np.float64)
    return np.exp(-((yy - c) ** 2 + (xx - c) ** 2) / (2 * s * s)).astype(np.complex64)


def raster_offsets(n: int, m: int, step: int, jitter: int = 0, seed: int = 0,
                   n_cols: int | None = None) -> np.ndarray:
    """(J, 2) int32 top-left (row, col) offsets of a jittered raster scan, row-major."""
    W = n if n_cols is None else n_cols
    kr = (n - m) // step + 1
    kc = (W - m) // step + 1
    rows = np.arange(kr) * step
    cols = np.arange(kc) * step
    oo = np.stack(np.meshgrid(rows, cols, indexing="ij"), -1).reshape(-1, 2).astype(np.int64)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        jit = rng.integers(-jitter, jitter + 1, size=oo.shape)
        ia, ib = np.meshgrid(np.arange(kr), np.arange(kc), indexing="ij")
        ia, ib = ia.reshape(-1), ib.reshape(-1)
        jit[(ia == 0) | (ia == kr - 1), 0] = 0
        jit[(ib == 0) | (ib == kc - 1), 1] = 0
        oo = oo + jit
        oo[:, 0] = np.clip(oo[:, 0], 0, n - m)
        oo[:, 1] = np.clip(oo[:, 1], 0, W - m)
    return oo.astype(np.int32)


def lit_mask(h: int, w: int, m: int, offsets: np.ndarray, radius: float | None = None) -> np.ndarray:
    """Pixels inside at least one probe disk (geometric coverage of the scan)."""
    R = probe_radius(m) if radius is None else float(radius)
    c = 0.5 * (m - 1)
    yy, xx = np.mgrid[0:m, 0:m].astype(np.float64)
    disk = ((yy - c) ** 2 + (xx - c) ** 2) <= R * R
    lit = np.zeros((h, w), bool)
    for r0, c0 in np.asarray(offsets):
        lit[r0:r0 + m, c0:c0 + m] |= disk
    return lit


def make_truth(n: int, m: int, offsets: np.ndarray, seed: int, radius: float | None = None) -> np.ndarray:
    u = make_image(n, seed)
    u[~lit_mask(n, n, m, offsets, radius)] = 1.0
    return u


def poissonize(f_clean: np.ndarray, peak: float | None, seed: int) -> np.ndarray:
    """Poisson counts at `peak` photons for the brightest pixel, scaled back (FP32)."""
    f_clean = np.asarray(f_clean, np.float64)
    if peak is None:
        return f_clean.astype(np.float32)
    kappa = float(peak) / float(f_clean.max())
    rng = np.random.default_rng(seed)
    return (rng.poisson(kappa * f_clean) / kappa).astype(np.float32)


@dataclasses.dataclass
class Problem:
    """One synthetic reconstruction problem (sizes, scan, parameters)."""
    name: str
    n: int
    m: int
    step: int
    jitter: int
    sub_rows: int
    sub_cols: int
    overlap_px: int
    peak: float | None
    n_iter: int
    eps: float = 0.5
    eta: float = 0.1
    r: float = 0.05
    blind: bool = False
    mu: float = 0.0
    gamma: float = 0.0
    seed: int = 1

    def offsets(self) -> np.ndarray:
        return raster_offsets(self.n, self.m, self.step, self.jitter, seed=self.seed + 1000)

    def truth(self) -> np.ndarray:
        return make_truth(self.n, self.m, self.offsets(), self.seed)

    def probe(self) -> np.ndarray:
        return make_probe(self.m)


# The five workloads, sized as stated for this build (sections 4.1-4.2 give
# the paper's own: 256^2 / 512^2 samples, 64^2 probe, steps 8-16, D up to 10).
def small_2sub() -> Problem:
    """64^2 image, 16^2 probe, step 4 (169 frames), 2 column subdomains, noiseless, 50 its."""
    return Problem("od2p_64px_m16_2sub", 64, 16, 4, 0, 1, 2, 8, None, 50)


def grid_4x4() -> Problem:
    """512^2 image, 64^2 probe, step 16 +-2 jitter (841 frames), 4x4 subdomains, Poisson 1e4, 200 its."""
    return Problem("od2p_512px_m64_4x4", 512, 64, 16, 2, 4, 4, 16, 1e4, 200, eta=2.0, r=0.5)


def blind_4x4() -> Problem:
    """1024^2 image, 128^2 probe, step 32 +-3 (841 frames), 4x4 blind, Poisson 1e4."""
    return Problem("od2bp_1024px_m128_4x4", 1024, 128, 32, 3, 4, 4, 32, 1e4, 100, blind=True)


def large_blind() -> Problem:
    """4096^2 image, 256^2 probe, step 48 +-4 (6561 frames), 8x8 blind, Poisson 1e5."""
    return Problem("od2bp_4096px_m256_8x8", 4096, 256, 48, 4, 8, 8, 64, 1e5, 100, blind=True)


def batched_problems(count: int = 64, seed: int = 3) -> list[Problem]:
    """Heterogeneous independent reconstructions: N in [256, 1024], m in {32, 64, 128},
    step in [8, m/2], G x G subdomains with 2 <= G <= 8, Poisson peak 1e3..1e5.
    N is snapped to m + (k-1) step so that the raster tiles the image exactly."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(rng.choice([32, 64, 128]))
        step = int(rng.integers(8, m // 2 + 1))
        n0 = int(rng.integers(256, 1025))
        k = max(2, (n0 - m) // step + 1)
        while m + (k - 1) * step < 256:
            k += 1
        n = m + (k - 1) * step
        g = int(rng.integers(2, min(8, k) + 1))
        peak = float(10 ** rng.uniform(3, 5))
        out.append(Problem(f"batch{i}", n, m, step, 0, g, g, 16, peak, 50, seed=seed * 1000 + i))
    return out
