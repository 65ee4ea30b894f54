"""ctypes binding of libod2p.so (the C ABI of include/od2p.h).

Loading fails loudly when the library has not been built: there is no CPU or
PyTorch fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libod2p.so")

_lock = threading.Lock()
_lib = None

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_STATE = range(7)
STATE_U, STATE_GAMMA, STATE_LAMBDA, STATE_WD, STATE_DELTA, STATE_W, STATE_Q = range(7)
OA_IFFT = 1
LAUNCH_VARIANTS = 2

# Every symbol declared in include/od2p.h: (restype, argtypes)
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_F = ctypes.c_float


class Geometry(ctypes.Structure):
    """Mirror of ptycho_geometry."""
    _fields_ = [
        ("img_h", _I32), ("img_w", _I32), ("m", _I32), ("n_frames", _I32),
        ("offsets_host", _P), ("sub_rows", _I32), ("sub_cols", _I32), ("overlap_px", _I32),
        ("eps", _F), ("eta", _F), ("r", _F), ("mu", _F), ("gamma", _F), ("blind", _I32),
        ("fourier_support_host", _P), ("periodic", _I32),
    ]


SIGNATURES = {
    "ptycho_last_error": (ctypes.c_char_p, []),
    "ptycho_abi_version": (_I32, []),
    "ptycho_release_cached_memory": (ctypes.c_int, []),
    "ptycho_plan": (ctypes.c_int, [_P, ctypes.POINTER(Geometry), _P, _P]),
    "ptycho_plan_destroy": (ctypes.c_int, [_P]),
    "ptycho_decompose": (ctypes.c_int, [ctypes.POINTER(Geometry), _P, _P]),
    "ptycho_plan_shard": (ctypes.c_int, [_P, ctypes.POINTER(Geometry), _P, _I32, _P, _P]),
    "ptycho_plan_frames": (ctypes.c_int, [_P, _P, _P]),
    "od2p_halo_size": (ctypes.c_int, [_P, _I32, _P, _P]),
    "od2p_halo_pack": (ctypes.c_int, [_P, _I32, _P, _P]),
    "od2p_halo_unpack": (ctypes.c_int, [_P, _I32, _P, _P]),
    "ptycho_plan_dims": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "ptycho_plan_layout": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "ptycho_plan_periodic_layout": (ctypes.c_int, [_P, _P, _P]),
    "ptycho_forward": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "stagm_prox": (ctypes.c_int, [_P, _P, _P, _I64, _F, _F, _P]),
    "overlap_add": (ctypes.c_int, [_P, _P, _P, _P, _I32, _P]),
    "od2p_init": (ctypes.c_int, [_P, _P, _P, _P]),
    "od2p_iterate": (ctypes.c_int, [_P, _I32, _P]),
    "od2p_frame_update": (ctypes.c_int, [_P, _P]),
    "od2p_subdomain_update": (ctypes.c_int, [_P, _P]),
    "probe_update": (ctypes.c_int, [_P, _P]),
    "od2p_merge": (ctypes.c_int, [_P, _P, _P]),
    "od2p_metrics": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "od2p_state_len": (ctypes.c_int, [_P, _I32, _P]),
    "od2p_get_state": (ctypes.c_int, [_P, _I32, _P, _P]),
    "od2p_set_state": (ctypes.c_int, [_P, _I32, _P, _P]),
    "stagm_loss_grad": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _I32, _P]),
    "stagm_loss_noalloc": (ctypes.c_int, [_P, _I32, _I32, _P, _I32, _P, _I32, _P, _F, _P, _P]),
    "ptycho_batch_plan": (ctypes.c_int, [_P, _P, _P, _I32, _P]),
    "ptycho_batch_destroy": (ctypes.c_int, [_P]),
    "ptycho_batch_size": (ctypes.c_int, [_P, _P]),
    "ptycho_batch_member": (ctypes.c_int, [_P, _I32, _P]),
    "ptycho_batch_iterate": (ctypes.c_int, [_P, _I32, _P]),
    "ptycho_probe_init": (ctypes.c_int, [_P, _P, _P]),
    "od2p_set_penalties": (ctypes.c_int, [_P, _F, _F, _P]),
    "od2p_consensus_residual": (ctypes.c_int, [_P, _P, _P]),
    "od2p_snr": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "od2p_operator_norms": (ctypes.c_int, [_P, _P, _P]),
    "od2p_iterate_until": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_int32, _P, _P, _P]),
    "od2p_gamma_snapshot": (ctypes.c_int, [_P, _P]),
    "ptycho_plan_set_fft": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
    "ptycho_plan_get_fft": (ctypes.c_int, [_P, _P]),
    "od2p_frame_residual": (ctypes.c_int, [_P, _P, _P]),
    "ptycho_peak_probe": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "ptycho_plan_set_launch": (ctypes.c_int, [_P, _I32, _I32, _P]),
    "ptycho_plan_get_launch": (ctypes.c_int, [_P, _P, _P, _P]),
    "ptycho_plan_get_waves": (ctypes.c_int, [_P, _P, _P, _P]),
    "ptycho_plan_set_waves": (ctypes.c_int, [_P, _I32, _I32, _P]),
    "ptycho_batch_set_launch": (ctypes.c_int, [_P, _I32, _I32, _P]),
    "ptycho_batch_get_launch": (ctypes.c_int, [_P, _P, _P]),
}


class PtychoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[od2p error {code}] {msg}")
        self.code = code


def load(path: str | None = None):
    """Load libod2p.so and attach the signatures of every exported entry point."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"{p} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def check(rc: int) -> None:
    if rc != OK:
        raise PtychoError(rc, load().ptycho_last_error().decode(errors="replace"))
