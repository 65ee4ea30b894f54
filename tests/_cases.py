"""Shared construction of seeded test problems (inputs from synth, intensities
from the FP64 oracle's forward operator, Poisson noise from synth)."""
import json
import os

import numpy as np

import oracle
from paper_2011_00162_gb300 import synth


def make_case(p: synth.Problem, noise_seed: int = 7):
    offs = p.offsets()
    u_true = p.truth()
    w = p.probe()
    f_clean = np.abs(oracle.forward(u_true, w, offs)) ** 2
    f = synth.poissonize(f_clean, p.peak, noise_seed)
    return offs, u_true, w, f


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.complex128).reshape(-1)
    b = np.asarray(b, np.complex128).reshape(-1)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def phase_aligned_rel(x, ref) -> float:
    """Relative L2 error after removing the global phase (section 4 compares up to it)."""
    x = np.asarray(x, np.complex128).reshape(-1)
    ref = np.asarray(ref, np.complex128).reshape(-1)
    th = np.angle(np.vdot(x, ref))
    return float(np.linalg.norm(x * np.exp(1j * th) - ref) / np.linalg.norm(ref))


def record(test: str, **figures) -> None:
    """Append the parity figures a test measured to the JSON-lines file named by
    $OD2P_PARITY_RECORD (nothing happens when it is unset)."""
    path = os.environ.get("OD2P_PARITY_RECORD")
    if not path:
        return
    with open(path, "a") as fh:
        fh.write(json.dumps({"test": test, **{k: ([float(x) for x in v] if isinstance(v, (list, tuple)) else float(v))
                                              for k, v in figures.items()}}) + "\n")
