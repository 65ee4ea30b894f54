"""Python binding of the C ABI with the same names (argument marshalling only).

Every function takes and returns CUDA tensors (complex64 for complex data,
float32 for intensities) and enqueues its work on the current PyTorch CUDA
stream.  All arithmetic runs in libod2p.so; nothing here computes any step of
the method, and there is no CPU path: a CPU tensor or a missing library raises.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np
import torch

from . import _lib
from ._lib import (OA_IFFT, STATE_DELTA, STATE_GAMMA, STATE_LAMBDA, STATE_Q, STATE_U, STATE_W,
                   STATE_WD, PtychoError, check)

__all__ = [
    "Geometry", "Plan", "ptycho_plan", "ptycho_forward", "stagm_prox", "overlap_add", "od2p_init",
    "od2p_iterate", "od2p_frame_update", "od2p_subdomain_update", "probe_update", "od2p_merge",
    "od2p_metrics", "od2p_state_len", "od2p_get_state", "od2p_set_state", "stagm_loss_grad", "PtychoError",
    "STATE_U", "STATE_GAMMA", "STATE_LAMBDA", "STATE_WD", "STATE_DELTA", "STATE_W", "STATE_Q",
    "Batch", "ptycho_batch_plan", "ptycho_batch_iterate", "ptycho_plan_set_launch", "ptycho_plan_get_launch",
    "ptycho_plan_get_waves", "ptycho_plan_set_waves",
    "ptycho_batch_set_launch", "ptycho_batch_get_launch", "LAUNCH_VARIANTS", "ptycho_probe_init",
    "ptycho_release_cached_memory", "od2p_set_penalties", "od2p_consensus_residual", "od2p_snr", "od2p_operator_norms", "ptycho_peak_probe",
           "od2p_iterate_until", "od2p_gamma_snapshot", "od2p_frame_residual", "ptycho_plan_set_fft",
           "ptycho_plan_get_fft",
           "PROBE_FMA", "PROBE_SMEM", "ptycho_decompose", "ptycho_plan_shard", "ptycho_plan_frames",
           "od2p_halo_size", "od2p_halo_pack", "od2p_halo_unpack", "RECOMPUTE", "STORE", "FROM_STORE",
]

LAUNCH_VARIANTS = _lib.LAUNCH_VARIANTS


def _stream(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None, dtype: torch.dtype, what: str) -> ctypes.c_void_p | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor (there is no CPU path)")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


@dataclasses.dataclass
class Geometry:
    """Problem description (mirror of ptycho_geometry)."""
    img_h: int
    img_w: int
    m: int
    offsets: np.ndarray          # (J, 2) int32 top-left (row, col)
    sub_rows: int = 1
    sub_cols: int = 1
    overlap_px: int = 0
    eps: float = 0.5
    eta: float = 0.1
    r: float = 0.05
    mu: float = 0.0
    gamma: float = 0.0
    blind: bool = False
    fourier_support: np.ndarray | None = None  # (m, m) uint8, blind only
    periodic: bool = False                     # windows wrap around the image (a torus)

    @property
    def n_frames(self) -> int:
        return int(np.asarray(self.offsets).reshape(-1, 2).shape[0])


class Plan:
    """Owns a ptycho_plan_t; freed by close() or garbage collection.  With
    `owner` (one rank per subdomain) it is the shard of rank `rank`, and f
    holds only that shard's frames (see ptycho_plan_shard)."""

    def __init__(self, geom: Geometry, f: torch.Tensor, stream=None, owner=None, rank: int = 0):
        self._lib = _lib.load()
        self.geom = geom
        self._offs = np.ascontiguousarray(np.asarray(geom.offsets, np.int32).reshape(-1, 2))
        self._mask = (np.ascontiguousarray(np.asarray(geom.fourier_support, np.uint8))
                      if geom.fourier_support is not None else None)
        J = self._offs.shape[0]
        g = _lib.Geometry(geom.img_h, geom.img_w, geom.m, J, self._offs.ctypes.data, geom.sub_rows,
                          geom.sub_cols, geom.overlap_px, geom.eps, geom.eta, geom.r, geom.mu,
                          geom.gamma, int(bool(geom.blind)),
                          self._mask.ctypes.data if self._mask is not None else None, int(bool(geom.periodic)))
        h = ctypes.c_void_p()
        if owner is None:
            if tuple(f.shape) != (J, geom.m, geom.m):
                raise ValueError(f"f must be (J, m, m) = {(J, geom.m, geom.m)}, got {tuple(f.shape)}")
            check(self._lib.ptycho_plan(ctypes.byref(h), ctypes.byref(g), _ptr(f, torch.float32, "f"),
                                        _stream(stream)))
        else:
            own = np.ascontiguousarray(np.asarray(owner, np.int32).reshape(-1))
            fs, _ = ptycho_decompose(geom)
            Js = int(np.count_nonzero(own[fs] == rank))
            if tuple(f.shape) != (Js, geom.m, geom.m):
                raise ValueError(f"f must hold the shard's {Js} frames, got {tuple(f.shape)}")
            check(self._lib.ptycho_plan_shard(ctypes.byref(h), ctypes.byref(g), own.ctypes.data, int(rank),
                                              _ptr(f, torch.float32, "f"), _stream(stream)))
            J = Js
        self.owner = None if owner is None else [int(x) for x in np.asarray(owner).reshape(-1)]
        self.rank = int(rank)
        self._h = h
        self.device = f.device
        D, P = ctypes.c_int32(), ctypes.c_int32()
        ul, ll = ctypes.c_int64(), ctypes.c_int64()
        check(self._lib.ptycho_plan_dims(h, ctypes.byref(D), ctypes.byref(P), ctypes.byref(ul),
                                         ctypes.byref(ll)))
        self.n_sub, self.n_pairs, self.u_len, self.lambda_len = D.value, P.value, ul.value, ll.value
        self.n_frames = J

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("plan has been destroyed")
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            self._lib.ptycho_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layout(self):
        """(frame_sub[J], rect[D,4], pair[P,2], pair_rect[P,4]) as numpy int32."""
        fs = np.empty(self.n_frames, np.int32)
        rect = np.empty((self.n_sub, 4), np.int32)
        pr = np.empty((max(self.n_pairs, 1), 2), np.int32)
        prc = np.empty((max(self.n_pairs, 1), 4), np.int32)
        check(self._lib.ptycho_plan_layout(self.handle, fs.ctypes.data, rect.ctypes.data,
                                           pr.ctypes.data, prc.ctypes.data))
        return fs, rect, pr[:self.n_pairs], prc[:self.n_pairs]

    def periodic_layout(self):
        """(pair_shift[P,2] in periods, placed offsets[J,2] in extended coordinates)."""
        sh = np.empty((max(self.n_pairs, 1), 2), np.int32)
        placed = np.empty((self.n_frames, 2), np.int32)
        check(self._lib.ptycho_plan_periodic_layout(self.handle, sh.ctypes.data, placed.ctypes.data))
        return sh[:self.n_pairs], placed


def ptycho_plan(geom: Geometry, f: torch.Tensor, stream=None) -> Plan:
    return Plan(geom, f, stream)


def ptycho_decompose(geom: Geometry):
    """(frame_sub[J], rect[D, 4]) of the decomposition, computed on the host."""
    g, keep = _geometry_struct(geom)
    fs = np.empty(geom.n_frames, np.int32)
    rect = np.empty((geom.sub_rows * geom.sub_cols, 4), np.int32)
    check(_lib.load().ptycho_decompose(ctypes.byref(g), fs.ctypes.data, rect.ctypes.data))
    del keep
    return fs, rect


def ptycho_plan_shard(geom: Geometry, owner, rank: int, f: torch.Tensor, stream=None) -> Plan:
    """The shard of rank `rank` (owner[d] = rank of subdomain d); f: its own frames."""
    return Plan(geom, f, stream, owner=owner, rank=rank)


def ptycho_plan_frames(plan: Plan) -> np.ndarray:
    """Global indices of the plan's frames."""
    out = np.empty(plan.n_frames, np.int32)
    check(plan._lib.ptycho_plan_frames(plan.handle, None, out.ctypes.data))
    return out


def od2p_halo_size(plan: Plan, peer: int) -> tuple[int, int]:
    a, b = ctypes.c_int64(), ctypes.c_int64()
    check(plan._lib.od2p_halo_size(plan.handle, int(peer), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def od2p_halo_pack(plan: Plan, peer: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    n, _ = od2p_halo_size(plan, peer)
    if out is None:
        out = torch.empty(n, dtype=torch.complex64, device=plan.device)
    if out.numel() != n:
        raise ValueError(f"send buffer must hold {n} complex values")
    check(plan._lib.od2p_halo_pack(plan.handle, int(peer), _ptr(out, torch.complex64, "out") if n else None,
                                   _stream(stream)))
    return out


def od2p_halo_unpack(plan: Plan, peer: int, msg: torch.Tensor, stream=None) -> None:
    _, n = od2p_halo_size(plan, peer)
    if msg.numel() != n:
        raise ValueError(f"message must hold {n} complex values")
    check(plan._lib.od2p_halo_unpack(plan.handle, int(peer), _ptr(msg, torch.complex64, "msg") if n else None,
                                     _stream(stream)))


def _geometry_struct(geom: Geometry):
    offs = np.ascontiguousarray(np.asarray(geom.offsets, np.int32).reshape(-1, 2))
    mask = (np.ascontiguousarray(np.asarray(geom.fourier_support, np.uint8))
            if geom.fourier_support is not None else None)
    g = _lib.Geometry(geom.img_h, geom.img_w, geom.m, offs.shape[0], offs.ctypes.data, geom.sub_rows,
                      geom.sub_cols, geom.overlap_px, geom.eps, geom.eta, geom.r, geom.mu, geom.gamma,
                      int(bool(geom.blind)), mask.ctypes.data if mask is not None else None,
                      int(bool(geom.periodic)))
    return g, (offs, mask)


class _Member(Plan):
    """A plan owned by a Batch (not destroyed by the wrapper)."""

    def __init__(self, handle, geom: Geometry, device):
        self._lib = _lib.load()
        self.geom = geom
        self._h = handle
        self.device = device
        D, P = ctypes.c_int32(), ctypes.c_int32()
        ul, ll = ctypes.c_int64(), ctypes.c_int64()
        check(self._lib.ptycho_plan_dims(handle, ctypes.byref(D), ctypes.byref(P), ctypes.byref(ul),
                                         ctypes.byref(ll)))
        self.n_sub, self.n_pairs, self.u_len, self.lambda_len = D.value, P.value, ul.value, ll.value
        self.n_frames = geom.n_frames

    def close(self) -> None:
        self._h = None  # the batch owns the plan


class Batch:
    """Independent nonblind reconstructions iterated together (ptycho_batch_*)."""

    def __init__(self, geoms: list, fs: list, stream=None):
        if len(geoms) != len(fs) or not geoms:
            raise ValueError("need matching, non-empty lists of geometries and intensity stacks")
        self._lib = _lib.load()
        structs, self._keep = [], []
        for g, f in zip(geoms, fs):
            st, keep = _geometry_struct(g)
            structs.append(st)
            self._keep.append(keep)
            if tuple(f.shape) != (g.n_frames, g.m, g.m):
                raise ValueError("each f must be (J, m, m)")
        arr = (_lib.Geometry * len(geoms))(*structs)
        ptrs = (ctypes.c_void_p * len(fs))(*[_ptr(f, torch.float32, "f").value for f in fs])
        h = ctypes.c_void_p()
        check(self._lib.ptycho_batch_plan(ctypes.byref(h), arr, ptrs, len(geoms), _stream(stream)))
        self._h = h
        self.members = []
        for i, g in enumerate(geoms):
            mp = ctypes.c_void_p()
            check(self._lib.ptycho_batch_member(h, i, ctypes.byref(mp)))
            self.members.append(_Member(mp, g, fs[i].device))

    def iterate(self, n_iter: int = 1, stream=None) -> None:
        check(self._lib.ptycho_batch_iterate(self._h, int(n_iter), _stream(stream)))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            for m in self.members:
                m._h = None
            self._lib.ptycho_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ptycho_batch_plan(geoms: list, fs: list, stream=None) -> Batch:
    return Batch(geoms, fs, stream)


def ptycho_batch_iterate(batch: Batch, n_iter: int = 1, stream=None) -> None:
    batch.iterate(n_iter, stream)


def od2p_set_penalties(plan: Plan, eta: float, r: float, stream=None) -> None:
    """Change the penalties for the next iterations, keeping eta*Gamma and r*Lambda."""
    check(plan._lib.od2p_set_penalties(plan.handle, float(eta), float(r), _stream(stream)))
    plan.geom = dataclasses.replace(plan.geom, eta=float(eta), r=float(r))


def od2p_consensus_residual(plan: Plan, stream=None) -> float:
    """||u_d - u_e|| over the pairs' overlaps relative to ||u||."""
    v = ctypes.c_float()
    check(plan._lib.od2p_consensus_residual(plan.handle, ctypes.byref(v), _stream(stream)))
    return v.value


def od2p_snr(plan: Plan, truth: torch.Tensor, mask: torch.Tensor | None = None, stream=None) -> float:
    """Section 4's SNR (dB) of the merged recovery against the ground truth
    (img_h x img_w), over the pixels where `mask` (bool/uint8, same shape) is set."""
    g = plan.geom
    if tuple(truth.shape) != (g.img_h, g.img_w):
        raise ValueError("truth must be (img_h, img_w)")
    mp = None
    if mask is not None:
        if tuple(mask.shape) != (g.img_h, g.img_w):
            raise ValueError("mask must be (img_h, img_w)")
        mask = mask.to(torch.uint8).contiguous()
        mp = _ptr(mask, torch.uint8, "mask")
    v = ctypes.c_float()
    check(plan._lib.od2p_snr(plan.handle, _ptr(truth.contiguous(), torch.complex64, "truth"), mp,
                             ctypes.byref(v), _stream(stream)))
    return v.value


def od2p_operator_norms(plan: Plan, stream=None) -> tuple[float, float]:
    """(max_d ||A_d^* A_d||, max_(d,e) ||pi_{d,e} A_d^*||^2) of a nonblind plan (Lemma 2.4)."""
    v = (ctypes.c_float * 2)()
    check(plan._lib.od2p_operator_norms(plan.handle, v, _stream(stream)))
    return float(v[0]), float(v[1])


PROBE_FMA, PROBE_SMEM = 0, 1


def ptycho_peak_probe(kind: int, n_blocks: int, iters: int, sink: torch.Tensor, stream=None) -> None:
    """Launch the FP32-FMA (PROBE_FMA) or shared-memory (PROBE_SMEM) throughput
    probe: n_blocks x 256 threads; sink holds n_blocks * 256 floats."""
    if sink.numel() < n_blocks * 256:
        raise ValueError("sink must hold n_blocks * 256 floats")
    check(_lib.load().ptycho_peak_probe(int(kind), int(n_blocks), int(iters), _ptr(sink, torch.float32, "sink"),
                                        _stream(stream)))


def od2p_iterate_until(plan: Plan, rf_tol: float, max_iter: int, stream=None) -> tuple[int, float]:
    """Iterate until (float) RF <= rf_tol or max_iter iterations, the test
    evaluated on the device after every iteration; returns (iterations, RF)."""
    n = ctypes.c_int32()
    rf = ctypes.c_float()
    check(plan._lib.od2p_iterate_until(plan.handle, float(rf_tol), int(max_iter), ctypes.byref(n),
                                       ctypes.byref(rf), _stream(stream)))
    return int(n.value), float(rf.value)


def od2p_gamma_snapshot(plan: Plan, stream=None) -> None:
    """Keep a copy of Gamma for od2p_frame_residual."""
    check(plan._lib.od2p_gamma_snapshot(plan.handle, _stream(stream)))


def od2p_frame_residual(plan: Plan, stream=None) -> float:
    """||Gamma - Gamma_snapshot|| / ||sqrt f||: the frame constraint's relative primal residual."""
    v = ctypes.c_float()
    check(plan._lib.od2p_frame_residual(plan.handle, ctypes.byref(v), _stream(stream)))
    return v.value


def ptycho_plan_set_fft(plan: Plan, kind: int, stream=None) -> None:
    """m = 64: 0 = the 8 x 8 transform split, 1 / 2 = the 16 x 4 split (Gamma staged / via L2)."""
    check(plan._lib.ptycho_plan_set_fft(plan.handle, int(kind), _stream(stream)))


def ptycho_plan_get_fft(plan: Plan) -> int:
    k = ctypes.c_int32()
    check(plan._lib.ptycho_plan_get_fft(plan.handle, ctypes.byref(k)))
    return int(k.value)


def ptycho_release_cached_memory() -> None:
    """Return the plan memory pool's unused device memory to the driver."""
    check(_lib.load().ptycho_release_cached_memory())


def ptycho_probe_init(plan: Plan, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """w0 = (1/J) sum_j F^* sqrt(f_j) (m x m complex64) from the plan's intensities."""
    m = plan.geom.m
    if out is None:
        out = _c64((m, m), plan.device)
    check(plan._lib.ptycho_probe_init(plan.handle, _ptr(out, torch.complex64, "w0"), _stream(stream)))
    return out


def ptycho_plan_set_launch(plan: Plan, variant: int, blocks_per_sm: int = 0, stream=None) -> None:
    check(plan._lib.ptycho_plan_set_launch(plan.handle, int(variant), int(blocks_per_sm), _stream(stream)))


def ptycho_plan_get_launch(plan: Plan) -> tuple[int, int, int]:
    """(variant, blocks_per_sm cap (0: none), most blocks of this variant that fit per SM)."""
    v, b, mx = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    check(plan._lib.ptycho_plan_get_launch(plan.handle, ctypes.byref(v), ctypes.byref(b), ctypes.byref(mx)))
    return v.value, b.value, mx.value


def ptycho_plan_set_waves(plan: Plan, wave_frames: int, chains: int, stream=None) -> None:
    """m = 256: frames per wave and chains of waves side by side (same iterates for every shape)."""
    check(plan._lib.ptycho_plan_set_waves(plan.handle, int(wave_frames), int(chains), _stream(stream)))


def ptycho_plan_get_waves(plan: Plan) -> tuple[int, int, int]:
    """(frames per wave, chains of waves side by side, kernel launches of one frame update)."""
    wf, ch, ln = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    check(plan._lib.ptycho_plan_get_waves(plan.handle, ctypes.byref(wf), ctypes.byref(ch), ctypes.byref(ln)))
    return wf.value, ch.value, ln.value


def ptycho_batch_set_launch(batch: Batch, variant: int, blocks_per_sm: int = 0, stream=None) -> None:
    check(batch._lib.ptycho_batch_set_launch(batch._h, int(variant), int(blocks_per_sm), _stream(stream)))


def ptycho_batch_get_launch(batch: Batch) -> tuple[int, int]:
    v, b = ctypes.c_int32(), ctypes.c_int32()
    check(batch._lib.ptycho_batch_get_launch(batch._h, ctypes.byref(v), ctypes.byref(b)))
    return v.value, b.value


def _c64(shape, device):
    return torch.empty(shape, dtype=torch.complex64, device=device)


def ptycho_forward(plan: Plan, u: torch.Tensor, w: torch.Tensor, out: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    g = plan.geom
    if tuple(u.shape) != (g.img_h, g.img_w) or tuple(w.shape) != (g.m, g.m):
        raise ValueError("u must be (img_h, img_w) and w (m, m)")
    if out is None:
        out = _c64((plan.n_frames, g.m, g.m), u.device)
    check(plan._lib.ptycho_forward(plan.handle, _ptr(u, torch.complex64, "u"), _ptr(w, torch.complex64, "w"),
                                   _ptr(out, torch.complex64, "out"), _stream(stream)))
    return out


def stagm_prox(y: torch.Tensor, f: torch.Tensor, eps: float, lam: float,
               out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if y.shape != f.shape:
        raise ValueError("y and f must have the same shape")
    if out is None:
        out = torch.empty_like(y)
    check(_lib.load().stagm_prox(_ptr(y, torch.complex64, "y"), _ptr(f, torch.float32, "f"),
                                 _ptr(out, torch.complex64, "out"), y.numel(), eps, lam, _stream(stream)))
    return out


def overlap_add(plan: Plan, frames: torch.Tensor, w: torch.Tensor, ifft: bool = True,
                out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    g = plan.geom
    if tuple(frames.shape) != (plan.n_frames, g.m, g.m):
        raise ValueError("frames must be (J, m, m)")
    if out is None:
        out = _c64((g.img_h, g.img_w), frames.device)
    check(plan._lib.overlap_add(plan.handle, _ptr(frames, torch.complex64, "frames"),
                                _ptr(w, torch.complex64, "w"), _ptr(out, torch.complex64, "out"),
                                OA_IFFT if ifft else 0, _stream(stream)))
    return out


def od2p_init(plan: Plan, w0: torch.Tensor, u0: torch.Tensor | None = None, stream=None) -> None:
    check(plan._lib.od2p_init(plan.handle, _ptr(u0, torch.complex64, "u0"), _ptr(w0, torch.complex64, "w0"),
                              _stream(stream)))


def od2p_iterate(plan: Plan, n_iter: int = 1, stream=None) -> None:
    check(plan._lib.od2p_iterate(plan.handle, int(n_iter), _stream(stream)))


def od2p_frame_update(plan: Plan, stream=None) -> None:
    check(plan._lib.od2p_frame_update(plan.handle, _stream(stream)))


def od2p_subdomain_update(plan: Plan, stream=None) -> None:
    check(plan._lib.od2p_subdomain_update(plan.handle, _stream(stream)))


def probe_update(plan: Plan, stream=None) -> None:
    check(plan._lib.probe_update(plan.handle, _stream(stream)))


def od2p_merge(plan: Plan, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    g = plan.geom
    if out is None:
        out = _c64((g.img_h, g.img_w), plan.device)
    check(plan._lib.od2p_merge(plan.handle, _ptr(out, torch.complex64, "out"), _stream(stream)))
    return out


def od2p_metrics(plan: Plan, stream=None, loss: bool = False):
    """(RF, RE) of the last iteration; with loss=True also the ST-AGM loss of
    the current subdomain iterate: (RF, RE, loss)."""
    rf, re, ls = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    check(plan._lib.od2p_metrics(plan.handle, ctypes.byref(rf), ctypes.byref(re),
                                 ctypes.byref(ls) if loss else None, _stream(stream)))
    return (rf.value, re.value, ls.value) if loss else (rf.value, re.value)


def od2p_state_len(plan: Plan, which: int) -> int:
    n = ctypes.c_int64()
    check(plan._lib.od2p_state_len(plan.handle, int(which), ctypes.byref(n)))
    return n.value


def od2p_get_state(plan: Plan, which: int, stream=None) -> torch.Tensor:
    out = _c64((od2p_state_len(plan, which),), plan.device)
    check(plan._lib.od2p_get_state(plan.handle, int(which), _ptr(out, torch.complex64, "dst"), _stream(stream)))
    return out


def od2p_set_state(plan: Plan, which: int, src: torch.Tensor, stream=None) -> None:
    n = od2p_state_len(plan, which)
    if src.numel() != n:
        raise ValueError(f"state {which} has {n} elements, got {src.numel()}")
    check(plan._lib.od2p_set_state(plan.handle, int(which), _ptr(src.contiguous(), torch.complex64, "src"),
                                   _stream(stream)))


RECOMPUTE, STORE, FROM_STORE = 1, 0, 2  # stagm_loss_grad's recompute argument


def stagm_loss_grad(plan: Plan, u: torch.Tensor, w: torch.Tensor, grad_u: bool = True,
                    grad_w: bool = True, stream=None, recompute: int = RECOMPUTE):
    """(loss[1] float32, grad_u or None, grad_w or None) on the current stream;
    recompute = RECOMPUTE, STORE or FROM_STORE as in include/od2p.h."""
    g = plan.geom
    loss = torch.empty(1, dtype=torch.float32, device=u.device)
    gu = _c64((g.img_h, g.img_w), u.device) if grad_u else None
    gw = _c64((g.m, g.m), u.device) if grad_w else None
    check(plan._lib.stagm_loss_grad(plan.handle, _ptr(u, torch.complex64, "u"), _ptr(w, torch.complex64, "w"),
                                    _ptr(loss, torch.float32, "loss"), _ptr(gu, torch.complex64, "grad_u"),
                                    _ptr(gw, torch.complex64, "grad_w"), int(recompute), _stream(stream)))
    return loss, gu, gw
