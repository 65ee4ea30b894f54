"""FP64 CPU oracle for the OD2P ptychography iteration (arXiv:2011.00162).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It wraps the
plain-C double-precision library built from the ``*.c`` files next to this
file; the wrapper only marshals arrays.  It shares no code with the CUDA
library of ``paper_2011_00162_gb300``.

Every array crossing into C is converted to contiguous complex128 / float64 /
int32 first.  The functions follow the paper:

* :func:`fft2`, :func:`dft2`      -- the unitary DFT F (section 2);
* :func:`stagm_g`, :func:`stagm_grad`, :func:`stagm_prox` -- ST-AGM, its
  gradient and proximal map (section 2.2, eqs. obj-1, objgrad, Prox_sol);
* :func:`forward`, :func:`adjoint` -- A and A^* (section 2);
* :func:`loss_grad`               -- the ST-AGM data-fidelity loss and gradients;
* :func:`geometry`, :func:`pairs` -- the overlapping decomposition (sections 2.1, 3.1);
* :func:`operator_norms`          -- the norms in Lemma 2.4's parameter set K;
* :func:`probe_init`, :func:`snr` -- section 4.2's initial probe, section 4's SNR;
* :class:`ADMM`                   -- Algorithm 2 (nonblind) and Algorithm 3 (blind).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["fft.c", "stagm.c", "operator.c", "geometry.c", "admm.c"]
_LIBNAME = "liboracle.so"
_lock = threading.Lock()
_lib = None

U, GAMMA, LAMBDA, WD, DELTA, W, V, Z = range(8)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math) into oracle/liboracle.so."""
    out = os.path.join(_HERE, _LIBNAME)
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdr = os.path.join(_HERE, "od2p_oracle.h")
    if not force and os.path.exists(out):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr])
        if os.path.getmtime(out) >= newest:
            return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, out)
    return out


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        sig = {
            "orc_dft2": (None, [P, i32, i32]),
            "orc_fft2": (None, [P, i32, i32]),
            "orc_stagm_g_arr": (None, [P, P, i64, f64, P]),
            "orc_stagm_grad_arr": (None, [P, P, i64, f64, P]),
            "orc_stagm_prox_arr": (None, [P, P, i64, f64, f64, P]),
            "orc_forward": (None, [i32, i32, P, i32, P, i32, P, P]),
            "orc_adjoint": (None, [i32, i32, i32, P, i32, P, P, P]),
            "orc_loss_grad": (f64, [i32, i32, P, i32, P, i32, P, P, f64, P, P]),
            "orc_probe_init": (None, [i32, i32, P, P]),
            "orc_snr": (f64, [i64, P, P]),
            "orc_geometry": (i32, [i32, i32, i32, i32, P, i32, i32, i32, P, P]),
            "orc_pairs": (i32, [i32, P, i32, P, P]),
            "orc_forward_ext": (None, [i32, i32, P, i32, P, i32, P, i32, P]),
            "orc_adjoint_ext": (None, [i32, i32, i32, P, i32, P, i32, P, P]),
            "orc_loss_grad_ext": (f64, [i32, i32, P, i32, P, i32, P, i32, P, f64, P, P]),
            "orc_geometry_ext": (i32, [i32, i32, i32, i32, P, i32, i32, i32, i32, P, P, P]),
            "orc_pairs_ext": (i32, [i32, P, i32, i32, i32, i32, P, P, P]),
            "orc_admm_new_ext": (P, [i32, i32, i32, i32, P, i32, i32, i32, i32, P, P, P, f64, f64, f64,
                                     i32, f64, f64, P]),
            "orc_admm_new": (P, [i32, i32, i32, i32, P, i32, i32, i32, P, P, P, f64, f64, f64,
                                 i32, f64, f64, P]),
            "orc_admm_free": (None, [P]),
            "orc_admm_iterate": (None, [P, i32]),
            "orc_admm_num_sub": (i32, [P]),
            "orc_admm_num_pairs": (i32, [P]),
            "orc_admm_state_len": (i64, [P, i32]),
            "orc_admm_get": (None, [P, i32, P]),
            "orc_admm_set": (None, [P, i32, P]),
            "orc_admm_metrics": (None, [P, P, P]),
            "orc_admm_merge": (None, [P, P]),
            "orc_admm_set_penalties": (None, [P, f64, f64]),
            "orc_admm_consensus": (f64, [P]),
            "orc_admm_set_owned": (None, [P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def dft2(x, inverse: bool = False) -> np.ndarray:
    """Unitary 2-D DFT written out from its definition (O(m^4))."""
    x = _c(x, np.complex128).copy()
    _load().orc_dft2(_p(x), x.shape[-1], int(inverse))
    return x


def fft2(x, inverse: bool = False) -> np.ndarray:
    """Unitary 2-D radix-2 FFT of one m x m frame (m a power of two)."""
    x = _c(x, np.complex128).copy()
    _load().orc_fft2(_p(x), x.shape[-1], int(inverse))
    return x


def stagm_g(x, b, eps: float) -> np.ndarray:
    x = _c(x, np.complex128)
    b = _c(np.broadcast_to(b, x.shape), np.float64)
    out = np.empty(x.shape, np.float64)
    _load().orc_stagm_g_arr(_p(x), _p(b), x.size, eps, _p(out))
    return out


def stagm_grad(x, b, eps: float) -> np.ndarray:
    x = _c(x, np.complex128)
    b = _c(np.broadcast_to(b, x.shape), np.float64)
    out = np.empty(x.shape, np.complex128)
    _load().orc_stagm_grad_arr(_p(x), _p(b), x.size, eps, _p(out))
    return out


def stagm_prox(y, f, eps: float, lam: float) -> np.ndarray:
    y = _c(y, np.complex128)
    f = _c(np.broadcast_to(f, y.shape), np.float64)
    out = np.empty(y.shape, np.complex128)
    _load().orc_stagm_prox_arr(_p(y), _p(f), y.size, eps, lam, _p(out))
    return out


def forward(u, w, offs, periodic: bool = False) -> np.ndarray:
    """All frames F(w o S_j u), shape (J, m, m) (periodic: windows wrap)."""
    u = _c(u, np.complex128)
    w = _c(w, np.complex128)
    offs = _c(offs, np.int32).reshape(-1, 2)
    H, W = u.shape
    m = w.shape[0]
    out = np.empty((offs.shape[0], m, m), np.complex128)
    _load().orc_forward_ext(H, W, _p(u), m, _p(w), offs.shape[0], _p(offs), int(bool(periodic)), _p(out))
    return out


def adjoint(y, w, offs, H: int, W: int, periodic: bool = False) -> np.ndarray:
    """A^* y = sum_j S_j^T (conj(w) o F^* y_j), shape (H, W) (periodic: windows wrap)."""
    y = _c(y, np.complex128)
    w = _c(w, np.complex128)
    offs = _c(offs, np.int32).reshape(-1, 2)
    out = np.empty((H, W), np.complex128)
    _load().orc_adjoint_ext(H, W, w.shape[0], _p(w), offs.shape[0], _p(offs), int(bool(periodic)), _p(y), _p(out))
    return out


def loss_grad(u, w, offs, f, eps: float, periodic: bool = False):
    """(loss, grad_u, grad_w) of sum_j G_eps(F(w o S_j u); f_j) (periodic: windows wrap)."""
    u = _c(u, np.complex128)
    w = _c(w, np.complex128)
    f = _c(f, np.float64)
    offs = _c(offs, np.int32).reshape(-1, 2)
    H, W = u.shape
    gu = np.empty_like(u)
    gw = np.empty_like(w)
    loss = _load().orc_loss_grad_ext(H, W, _p(u), w.shape[0], _p(w), offs.shape[0], _p(offs),
                                     int(bool(periodic)), _p(f), eps, _p(gu), _p(gw))
    return float(loss), gu, gw


def probe_init(f) -> np.ndarray:
    """w0 = (1/J) sum_j F^* sqrt(f_j) (section 4.2's data-driven initial probe)."""
    f = _c(f, np.float64)
    J, m = f.shape[0], f.shape[-1]
    w0 = np.empty((m, m), np.complex128)
    _load().orc_probe_init(m, J, _p(f), _p(w0))
    return w0


def snr(ur, ug) -> float:
    """Section 4's SNR (dB) of the recovery ur against the ground truth ug
    (denominator ||ur||^2, as printed) after removing ur's global phase."""
    ur = _c(ur, np.complex128).reshape(-1)
    ug = _c(ug, np.complex128).reshape(-1)
    return float(_load().orc_snr(ur.size, _p(ur), _p(ug)))


def geometry(H: int, W: int, m: int, offs, sub_rows: int, sub_cols: int, overlap_px: int,
             periodic: bool = False, placed: bool = False):
    """(frame_sub[J], rect[D,4]) of the overlapping decomposition; with
    placed=True also the frames' offsets in extended coordinates (J, 2)."""
    offs = _c(offs, np.int32).reshape(-1, 2)
    J = offs.shape[0]
    fs = np.empty(max(J, 1), np.int32)
    rect = np.empty((sub_rows * sub_cols, 4), np.int32)
    ro = np.empty((max(J, 1), 2), np.int32)
    D = _load().orc_geometry_ext(H, W, m, J, _p(offs), sub_rows, sub_cols, overlap_px, int(bool(periodic)),
                                 _p(fs), _p(rect), _p(ro))
    if D < 0:
        raise ValueError(f"invalid geometry (code {D})")
    return (fs[:J], rect, ro[:J]) if placed else (fs[:J], rect)


def pairs(rect, H: int = 0, W: int = 0, periodic: bool = False, shifts: bool = False):
    """Ordered intersecting pairs (d, e) and their intersection rectangles (in
    d's coordinates); with shifts=True also each pair's shift s (periods)."""
    rect = _c(rect, np.int32).reshape(-1, 4)
    lib = _load()
    per = int(bool(periodic))
    n = lib.orc_pairs_ext(rect.shape[0], _p(rect), H, W, per, 0, None, None, None)
    pr = np.empty((max(n, 1), 2), np.int32)
    sh = np.empty((max(n, 1), 2), np.int32)
    prc = np.empty((max(n, 1), 4), np.int32)
    lib.orc_pairs_ext(rect.shape[0], _p(rect), H, W, per, n, _p(pr), _p(sh), _p(prc))
    return (pr[:n], sh[:n], prc[:n]) if shifts else (pr[:n], prc[:n])


def operator_norms(w, offs, H: int, W: int, sub_rows: int, sub_cols: int, overlap_px: int):
    """Lemma 2.4's operator norms over all subdomains and ordered overlap pairs:
    (max_d ||A_d^* A_d||, max_(d,e) ||pi_{d,e} A_d^*||^2).  A_d^* A_d is the
    diagonal of eq. (AtA): sum over the frames of subdomain d of S_j^T |w|^2."""
    w = _c(w, np.complex128)
    m = w.shape[0]
    offs = _c(offs, np.int32).reshape(-1, 2)
    fs, rect = geometry(H, W, m, offs, sub_rows, sub_cols, overlap_px)
    pr, prc = pairs(rect)
    illum = np.zeros((rect.shape[0], H, W))
    for j, (r0, c0) in enumerate(offs):
        illum[fs[j], r0:r0 + m, c0:c0 + m] += np.abs(w) ** 2
    a = max(illum[d, R[0]:R[2], R[1]:R[3]].max() for d, R in enumerate(rect))
    b = 0.0
    for (d, _e), P in zip(pr, prc):
        b = max(b, illum[d, P[0]:P[2], P[1]:P[3]].max())
    return float(a), float(b)


class ADMM:
    """Algorithm 2 (blind=False) or Algorithm 3 (blind=True) in FP64."""

    def __init__(self, f, w0, offs, H: int, W: int, sub_rows: int, sub_cols: int,
                 overlap_px: int, eps: float, eta: float, r: float, u0=None, blind: bool = False,
                 mu: float = 0.0, gamma: float = 0.0, mask=None, periodic: bool = False):
        self._lib = _load()
        f = _c(f, np.float64)
        w0 = _c(w0, np.complex128)
        offs = _c(offs, np.int32).reshape(-1, 2)
        u0c = _c(u0, np.complex128) if u0 is not None else None
        maskc = _c(mask, np.float64) if mask is not None else None
        self.m = w0.shape[0]
        self.J = offs.shape[0]
        self.H, self.W = H, W
        self._h = self._lib.orc_admm_new_ext(H, W, self.m, self.J, _p(offs), sub_rows, sub_cols,
                                             overlap_px, int(bool(periodic)), _p(f), _p(w0), _p(u0c), eps, eta,
                                             r, int(blind), mu, gamma, _p(maskc))
        if not self._h:
            raise ValueError("invalid ADMM geometry")
        self.D = self._lib.orc_admm_num_sub(self._h)
        self.P = self._lib.orc_admm_num_pairs(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_admm_free(h)
            self._h = None

    def set_penalties(self, eta: float, r: float) -> None:
        """Change eta and r, keeping the unscaled multipliers eta*Gamma and r*Lambda."""
        self._lib.orc_admm_set_penalties(self._h, float(eta), float(r))

    def set_owned(self, owned) -> None:
        """Update only the subdomains d with owned[d] != 0 (None: all of them);
        the others' u, Lambda, W_d and Delta_d are halo copies set from outside."""
        if owned is None:
            self._lib.orc_admm_set_owned(self._h, None)
            return
        o = _c(owned, np.int32).reshape(-1)
        if o.size != self.D:
            raise ValueError(f"ownership mask: expected {self.D} entries, got {o.size}")
        self._lib.orc_admm_set_owned(self._h, _p(o))

    def consensus(self) -> float:
        """||u_d - u_e|| over the pairs' overlaps relative to ||u||."""
        return float(self._lib.orc_admm_consensus(self._h))

    def iterate(self, n: int = 1) -> None:
        self._lib.orc_admm_iterate(self._h, int(n))

    def get(self, which: int) -> np.ndarray:
        n = self._lib.orc_admm_state_len(self._h, which)
        out = np.empty(n, np.complex128)
        self._lib.orc_admm_get(self._h, which, _p(out))
        return out

    def set(self, which: int, arr) -> None:
        n = self._lib.orc_admm_state_len(self._h, which)
        a = _c(arr, np.complex128).reshape(-1)
        if a.size != n:
            raise ValueError(f"state {which}: expected {n} elements, got {a.size}")
        self._lib.orc_admm_set(self._h, which, _p(a))

    def metrics(self):
        rf = ctypes.c_double()
        re = ctypes.c_double()
        self._lib.orc_admm_metrics(self._h, ctypes.byref(rf), ctypes.byref(re))
        return rf.value, re.value

    def merge(self) -> np.ndarray:
        out = np.empty((self.H, self.W), np.complex128)
        self._lib.orc_admm_merge(self._h, _p(out))
        return out
