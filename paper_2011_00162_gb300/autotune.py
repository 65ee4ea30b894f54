"""Autotuner for the launch shape of the frame update, with an on-disk cache.

The frame update (steps 1-3 of the OD2P iteration, section 3.1) is compiled in
two shapes per probe side (frames per block x threads per block, see
``ptycho_plan_set_launch`` in include/od2p.h), and its persistent grid can be
capped at fewer resident blocks per SM than fit.  Which combination is fastest
depends on the probe side, the number of frames and how the subdomain update
that follows shares the GPU, so it is measured: every candidate runs a few
whole ADMM iterations of the plan itself, timed with CUDA events on the
launching stream, and the fastest is kept and cached on disk under a key of
(GPU model, SM count, probe side, frames, subdomains, blind).

Every shape computes the same iterates bit for bit, so tuning over shapes never
changes a result: the plan's state is saved before the trials and restored
after them.  For m = 64 the tuner also times the 16 x 4 transform split
(``ptycho_plan_set_fft`` kinds 1 and 2) unless ``fft=False``: those kinds give
the same iterates up to FP32 rounding (tested against the FP64 oracle like the
default split), not bit for bit.

Cache file: ``$OD2P_AUTOTUNE_CACHE`` if set, else
``~/.cache/od2p/autotune.json``.  It is plain JSON; a missing or unreadable
file is treated as empty, and writes go through a temporary file and an atomic
rename.
"""
from __future__ import annotations

import json
import os
import tempfile

import torch

from . import api

CACHE_ENV = "OD2P_AUTOTUNE_CACHE"
CACHE_VERSION = 2


def cache_path() -> str:
    p = os.environ.get(CACHE_ENV)
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "od2p", "autotune.json")


def load_cache(path: str | None = None) -> dict:
    """Entries of the cache file ({} when it is missing, unreadable or of another version)."""
    path = path or cache_path()
    try:
        with open(path) as fh:
            doc = json.load(fh)
    except (OSError, ValueError):
        return {}
    if not isinstance(doc, dict) or doc.get("version") != CACHE_VERSION or not isinstance(doc.get("entries"), dict):
        return {}
    return doc["entries"]


def store_cache(key: str, entry: dict, path: str | None = None) -> None:
    """Add or replace one entry; the file is rewritten atomically."""
    path = path or cache_path()
    entries = load_cache(path)
    entries[key] = entry
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".autotune.", dir=d)
    try:
        with os.fdopen(fd, "w") as fh:
            json.dump({"version": CACHE_VERSION, "entries": entries}, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        try:
            os.unlink(tmp)
        except OSError:
            pass
        raise


def device_tag(device) -> str:
    props = torch.cuda.get_device_properties(device)
    return f"{props.name}|cc{props.major}{props.minor}|sm{props.multi_processor_count}"


def make_key(device_tag_: str, m: int, n_frames: int, n_sub: int, blind: bool, kind: str = "plan") -> str:
    return f"{kind}|{device_tag_}|m{m}|J{n_frames}|D{n_sub}|blind{int(bool(blind))}"


def candidates(max_per_sm: dict[int, int]) -> list[tuple[int, int]]:
    """(variant, blocks_per_sm) pairs to time: every cap from 1 up to what fits, per variant.

    max_per_sm maps variant -> the most resident blocks of that shape per SM.
    """
    out = []
    for v in sorted(max_per_sm):
        for b in range(max(1, max_per_sm[v]), 0, -1):
            out.append((v, b))
    return out


def _plan_key(plan: api.Plan) -> str:
    g = plan.geom
    return make_key(device_tag(plan.device), g.m, plan.n_frames, plan.n_sub, g.blind)


def _state_selectors(plan: api.Plan) -> list[int]:
    sel = [api.STATE_U, api.STATE_GAMMA, api.STATE_LAMBDA]
    if plan.geom.blind:
        sel += [api.STATE_WD, api.STATE_DELTA, api.STATE_W]
    return sel


def _time_iterations(run_one, n_iter: int, flush: torch.Tensor | None) -> float:
    """Median device time (us) of one call of run_one over n_iter calls."""
    s = torch.cuda.current_stream()
    times = []
    for _ in range(n_iter):
        if flush is not None:
            flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        run_one()
        b.record(s)
        b.synchronize()
        times.append(a.elapsed_time(b) * 1e3)
    times.sort()
    return times[len(times) // 2]


def _flush_buffer(device, flush_l2: bool):
    # larger than the 129 MB L2: every trial iteration starts from HBM
    return torch.empty(64 << 20, dtype=torch.float32, device=device) if flush_l2 else None


# m = 256, three passes: (frames per wave, chains side by side) tried by tune_plan
WAVE_SHAPES = [(19, 4), (38, 2), (12, 8), (16, 6), (28, 4)]


def _apply(plan: api.Plan, entry: dict) -> None:
    api.ptycho_plan_set_fft(plan, 0)
    api.ptycho_plan_set_launch(plan, int(entry["variant"]), int(entry["blocks_per_sm"]))
    if entry.get("fft", 0):
        api.ptycho_plan_set_fft(plan, int(entry["fft"]))
    if entry.get("waves"):
        api.ptycho_plan_set_waves(plan, int(entry["waves"][0]), int(entry["waves"][1]))


def tune_plan(plan: api.Plan, n_iter: int = 15, warmup: int = 3, flush_l2: bool = False, use_cache: bool = True,
              path: str | None = None, fft: bool = True) -> dict:
    """Pick and apply the fastest launch shape of plan's frame update.

    od2p_init must have been called.  flush_l2 writes a buffer larger than L2
    before every timed iteration (for callers that interleave other work with
    the iterations); by default iterations run back to back, as in a solve.
    Entries are cached per flush regime.  Returns the cache entry, with
    ``"cached": True`` when it came from the cache instead of a measurement.
    """
    fft = fft and plan.geom.m == 64
    key = _plan_key(plan) + ("|flush" if flush_l2 else "") + ("|fft" if fft else "")
    if use_cache:
        hit = load_cache(path).get(key)
        if hit is not None:
            _apply(plan, hit)
            return dict(hit, cached=True)
    saved = {w: api.od2p_get_state(plan, w).clone() for w in _state_selectors(plan)}
    maxes = {}
    for v in range(api.LAUNCH_VARIANTS):
        api.ptycho_plan_set_launch(plan, v, 0)
        maxes[v] = api.ptycho_plan_get_launch(plan)[2]
    flush = _flush_buffer(plan.device, flush_l2)
    trials = {}
    api.ptycho_plan_set_fft(plan, 0)
    # m = 256: the cluster launch against the three passes (no block cap)
    shapes_to_time = ([(v, 0) for v in range(api.LAUNCH_VARIANTS)] if plan.geom.m == 256
                      else candidates(maxes))
    for v, b in shapes_to_time:
        api.ptycho_plan_set_launch(plan, v, b)
        for _ in range(warmup):
            api.od2p_iterate(plan, 1)
        trials[f"{v}:{b}"] = _time_iterations(lambda: api.od2p_iterate(plan, 1), n_iter, flush)
    shapes = dict(trials)
    best_shape = min(shapes, key=shapes.get)
    v, b = (int(x) for x in best_shape.split(":"))
    api.ptycho_plan_set_launch(plan, v, b)
    waves = None
    if plan.geom.m == 256 and v == 0:  # the wave shape of the three passes
        wtrials = {}
        for wf, ch in WAVE_SHAPES:
            api.ptycho_plan_set_waves(plan, wf, ch)
            for _ in range(warmup):
                api.od2p_iterate(plan, 1)
            wtrials[f"waves{wf}x{ch}"] = _time_iterations(lambda: api.od2p_iterate(plan, 1), n_iter, flush)
        trials.update(wtrials)
        best_w = min(wtrials, key=wtrials.get)
        waves = [int(x) for x in best_w[5:].split("x")]
        api.ptycho_plan_set_waves(plan, *waves)
    for k in ((1, 2) if fft else ()):
        api.ptycho_plan_set_fft(plan, k)
        for _ in range(warmup):
            api.od2p_iterate(plan, 1)
        trials[f"fft{k}"] = _time_iterations(lambda: api.od2p_iterate(plan, 1), n_iter, flush)
    api.ptycho_plan_set_fft(plan, 0)
    best = min((k for k in trials if not k.startswith("waves")), key=trials.get)
    if waves:
        best = f"waves{waves[0]}x{waves[1]}"
    entry = {"variant": v, "blocks_per_sm": b, "fft": int(best[3:]) if best.startswith("fft") else 0,
             "us": trials[best], "trials": trials, "waves": waves}
    _apply(plan, entry)
    for w, t in saved.items():
        api.od2p_set_state(plan, w, t)
    torch.cuda.current_stream().synchronize()
    if use_cache:
        store_cache(key, entry, path)
    return dict(entry, cached=False)


def tune_batch(batch: api.Batch, n_iter: int = 15, warmup: int = 3, flush_l2: bool = False, use_cache: bool = True,
               path: str | None = None) -> dict:
    """Pick and apply the fastest launch shape of a batch's frame updates (as tune_plan)."""
    ms = sorted({mb.geom.m for mb in batch.members})
    frames = sum(mb.n_frames for mb in batch.members)
    subs = sum(mb.n_sub for mb in batch.members)
    key = make_key(device_tag(batch.members[0].device), max(ms), frames, subs, False,
                   kind=f"batch{len(batch.members)}m" + "-".join(map(str, ms))) + ("|flush" if flush_l2 else "")
    if use_cache:
        hit = load_cache(path).get(key)
        if hit is not None:
            api.ptycho_batch_set_launch(batch, int(hit["variant"]), int(hit["blocks_per_sm"]))
            return dict(hit, cached=True)
    saved = [{w: api.od2p_get_state(mb, w).clone() for w in _state_selectors(mb)} for mb in batch.members]
    maxes = {}
    for v in range(api.LAUNCH_VARIANTS):
        api.ptycho_batch_set_launch(batch, v, 0)
        maxes[v] = min(api.ptycho_plan_get_launch(mb)[2] for mb in batch.members)
    flush = _flush_buffer(batch.members[0].device, flush_l2)
    trials = {}
    for v, b in candidates(maxes):
        api.ptycho_batch_set_launch(batch, v, b)
        for _ in range(warmup):
            batch.iterate(1)
        trials[f"{v}:{b}"] = _time_iterations(lambda: batch.iterate(1), n_iter, flush)
    best = min(trials, key=trials.get)
    v, b = (int(x) for x in best.split(":"))
    api.ptycho_batch_set_launch(batch, v, b)
    for mb, st in zip(batch.members, saved):
        for w, t in st.items():
            api.od2p_set_state(mb, w, t)
    torch.cuda.current_stream().synchronize()
    entry = {"variant": v, "blocks_per_sm": b, "us": trials[best], "trials": trials}
    if use_cache:
        store_cache(key, entry, path)
    return dict(entry, cached=False)
