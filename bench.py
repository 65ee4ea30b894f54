"""Throughput of the OD2P iteration on GB300: ADMM frame-updates per second.

Headline workload (one step = one full ADMM iteration of Algorithm 3, the
blind OD2BP iteration, over all frames, replayed from its CUDA graph):
4096 x 4096 complex64 image, unknown 256 x 256 probe started from a Gaussian,
raster step 48 with +-4 px jitter (6561 frames, 1.72 GB of FP32 intensities),
8 x 8 subdomains with a 64 px minimum overlap, Poisson noise at 1e5 photons
peak -- the largest workload that fits one GPU.  Its per-iteration traffic
(about 12 GB) is far larger than the 129 MB L2, so no flush is needed between
timed iterations.  The 512 x 512 / 841-frame / 64 x 64 nonblind workload is
measured the same way (L2 flushed before each timed iteration, its working
set being L2-sized) and reported under "config2".

Inputs are seeded synthetic stand-ins for the paper's sample (section 4):
truth, probe and scan from paper_2011_00162_gb300.synth, and the measured
intensities simulated on the host from them with scipy's FFT and seeded
Poisson draws (simulate_intensities below), identically for both arms.

Timing: W untimed warm-up iterations, then K timed iterations, each bracketed
by CUDA events on the launch stream.  The roofline's kernel duration comes
from further iterations launched stage by stage (frame update, probe update,
subdomain update) with events around each.  Clocks are sampled with
nvidia-smi from before the timed region until after the stage timing.

`e2e` times the public API end to end with host buffers: pinned f copied to
the device, plan, Step 0, the workload's iterations, merge, image copied back
-- per reconstruction, frame-updates/s.

`--impl reference` times the FP64 CPU oracle (a plain restatement of the
paper) on a bounded sample of the same workload (a crop with the same probe,
step, jitter, noise and blind parameters), one oracle iteration per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "od2bp_4096px_m256_6561frames_8x8sub_poisson1e5"
WORKLOAD2 = "od2p_512px_m64_841frames_4x4sub_poisson1e4"
METRIC = "ADMM frame-updates/sec"
UNIT = "frame-updates/s"
BLIND_PRM = {"eta": 2.0, "r": 0.5, "mu": 1.0, "gamma": 0.1}
TRAFFIC_FILE_256 = os.path.join(ROOT, "profiles", "frame_update_m256_variant{variant}_2048px_1444frames.md")


def _problem():
    """The headline workload: blind, 4096^2, 6561 frames of 256^2, 8 x 8 subdomains."""
    import dataclasses

    from paper_2011_00162_gb300 import synth
    return dataclasses.replace(synth.large_blind(), eta=BLIND_PRM["eta"], r=BLIND_PRM["r"], mu=BLIND_PRM["mu"],
                               gamma=BLIND_PRM["gamma"])


def _problem2():
    from paper_2011_00162_gb300 import synth
    return synth.grid_4x4()


def simulate_intensities(p, seed: int = 7, chunk: int = 64) -> np.ndarray:
    """Measured intensities of problem p for the benchmark, on the host:
    f_clean = |F(w o S_j u)|^2 (unitary 2-D DFT, float64, scipy's FFT on all
    cores), then f = Poisson(kappa f_clean) / kappa with kappa = peak / max
    f_clean, drawn per chunk of 64 frames from numpy generators seeded
    (seed, chunk index) on a thread pool, returned as FP32 (J x m x m).  Both
    arms of this benchmark take their intensities from here."""
    from concurrent.futures import ThreadPoolExecutor
    try:
        import scipy.fft as sfft

        def fft2(x):
            return sfft.fft2(x, norm="ortho", workers=os.cpu_count() or 1)
    except ImportError:  # numpy's FFT, single-threaded
        def fft2(x):
            return np.fft.fft2(x, norm="ortho")
    offs = np.asarray(p.offsets())
    u = np.asarray(p.truth(), np.complex128)
    w = np.asarray(p.probe(), np.complex128)
    m, J = p.m, len(offs)
    f = np.empty((J, m, m), np.float32)
    clean = np.empty((J, m, m), np.float64)
    for j0 in range(0, J, chunk):
        j1 = min(J, j0 + chunk)
        psi = np.stack([w * u[r:r + m, c:c + m] for r, c in offs[j0:j1]])
        clean[j0:j1] = np.abs(fft2(psi)) ** 2
    if p.peak is None:
        f[:] = clean
        return f
    kappa = float(p.peak) / float(clean.max())

    def draw(k):
        j0, j1 = k * chunk, min(J, (k + 1) * chunk)
        rng = np.random.default_rng([seed, k])
        f[j0:j1] = rng.poisson(kappa * clean[j0:j1]) / kappa

    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        list(ex.map(draw, range((J + chunk - 1) // chunk)))
    return f


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"od2p_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        self.t0 = self.t1 = None
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        import datetime
        rows, all_rows = [], []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                row = (float(parts[2]), float(parts[3]), float(parts[4]) if parts[4] not in ("[N/A]", "") else 0.0,
                       parts[6:10])
            except ValueError:
                continue
            all_rows.append(row)
            if self.t0 is not None and self.t0 - 0.05 <= ts <= (self.t1 or ts) + 0.05:
                rows.append(row)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples in the timed region"],
                    "samples_outside": len(all_rows)}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        loaded = [r[0] for r in rows if r[2] > 200.0] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _geometry(od, p, offs, blind: bool):
    return od.Geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px, p.eps, p.eta, p.r,
                       mu=p.mu if blind else 0.0, gamma=p.gamma if blind else 0.0, blind=blind)


def _initial_probe(p, blind: bool) -> np.ndarray:
    from paper_2011_00162_gb300 import synth
    return synth.gaussian_probe(p.m) if blind else p.probe()


def _k1_launches(od, plan) -> int:
    """Kernel launches of one frame update, as the library reports them (m = 256,
    three-pass variant 0: three per wave; every other frame update is one)."""
    return od.ptycho_plan_get_waves(plan)[2]


def launches_per_iteration(od, plan) -> int:
    """Kernel launches of one graph-replayed ADMM iteration: the frame update,
    (blind) the probe average, the probe partial sums and the W/Delta update,
    and the subdomain update."""
    return _k1_launches(od, plan) + (3 if plan.geom.blind else 0) + 1


def e2e_run(od, geom, f, w0, offs, p, dev, ws, tune=True, n_e2e=3):
    """The public API end to end with host buffers, per reconstruction: pinned
    intensities and probe copied to the device, plan, Step 0, p.n_iter
    iterations, merge, the image copied back."""
    import torch
    from paper_2011_00162_gb300 import autotune
    f_pin = torch.from_numpy(f).pin_memory()
    w_pin = torch.from_numpy(w0).pin_memory()
    e2e_times = []
    out_host = torch.empty((p.n, p.n), dtype=torch.complex64).pin_memory()
    plan_s = None
    phases = {}
    for i in range(n_e2e + 2):
        # the last pass is not timed: it synchronises after every set-up phase to split them
        split = i == n_e2e + 1

        def mark(name):
            if split:
                torch.cuda.synchronize()
                phases[name] = round(1e3 * (time.perf_counter() - t0), 3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fd = f_pin.to(dev, non_blocking=True)
        wd = w_pin.to(dev, non_blocking=True)
        mark("h2d")
        pl = od.ptycho_plan(geom, fd)
        mark("plan")
        od.od2p_init(pl, wd)
        mark("init")
        if tune:
            autotune.tune_plan(pl)  # measured in the untimed first pass, a cache hit afterwards
        mark("tune")
        if i == 1:  # one extra synchronisation, to split the set-up from the iterations
            torch.cuda.synchronize()
            plan_s = time.perf_counter() - t0
        od.od2p_iterate(pl, p.n_iter)
        u = od.od2p_merge(pl)
        out_host.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        pl.close()
        del fd
        if 0 < i <= n_e2e:
            e2e_times.append(t1 - t0)
    value = len(offs) * p.n_iter * ws / statistics.median(e2e_times)
    return {"value": round(value, 1), "unit": UNIT,
            "h2d_bytes_per_step": int(f.nbytes + w0.nbytes),
            "d2h_bytes_per_step": int(out_host.numel() * 8),
            "step": f"one reconstruction: H2D f and w0, plan, init, {p.n_iter} iterations, merge, D2H image",
            "setup_ms": round(1e3 * plan_s, 3) if plan_s is not None else None,
            "setup_split_ms": {"cumulative, untimed pass": phases}}


def batched_leg(od, dev, K: int = 10, W: int = 2, count: int = 64, tune=True, retune=False):
    """Config-3 workload: `count` independent nonblind reconstructions of mixed
    sizes.  The batch (one frame-update launch per probe side + one subdomain
    update per iteration, graph-replayed) against the same plans iterated one
    after another, each plain plan on the transform split the batch uses (the
    16 x 4 split for m = 64, the two-stage split otherwise), so that equal
    error shows as bitwise-identical states."""
    import torch
    from paper_2011_00162_gb300 import synth
    probs = synth.batched_problems(count, seed=3)
    gen = torch.Generator(device=dev)
    gen.manual_seed(3)
    geoms, fs, ws = [], [], []
    for p in probs:
        offs = p.offsets()
        u, w = p.truth(), p.probe()
        tmp = od.ptycho_plan(od.Geometry(p.n, p.n, p.m, offs),
                             torch.ones((len(offs), p.m, p.m), dtype=torch.float32, device=dev))
        fr = od.ptycho_forward(tmp, torch.from_numpy(u).to(dev), torch.from_numpy(w).to(dev))
        tmp.close()
        fc = fr.abs() ** 2
        kappa = float(p.peak) / float(fc.max())
        fs.append((torch.poisson(fc * kappa, generator=gen) / kappa).float().contiguous())
        ws.append(torch.from_numpy(w).to(dev))
        geoms.append(od.Geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px, 0.5, 2.0, 0.5))
        del fr, fc
    J = sum(g.n_frames for g in geoms)
    batch = od.ptycho_batch_plan(geoms, fs)
    for m, w in zip(batch.members, ws):
        od.od2p_init(m, w)
    plains = [od.ptycho_plan(g, f) for g, f in zip(geoms, fs)]
    for pl, w in zip(plains, ws):
        od.od2p_init(pl, w)
    if tune:
        from paper_2011_00162_gb300 import autotune
        autotune.tune_batch(batch, use_cache=not retune)
        for pl in plains:  # launch shapes only: the transform split stays the batch's
            autotune.tune_plan(pl, use_cache=not retune, fft=False)
    for pl in plains:  # the batch runs its m = 64 members on the 16 x 4 split (fft kind 2)
        if pl.geom.m == 64:
            od.ptycho_plan_set_fft(pl, 2)
    batch.iterate(W)
    for pl in plains:
        od.od2p_iterate(pl, W)
    s = torch.cuda.current_stream()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    e[0].record(s)
    batch.iterate(K)
    e[1].record(s)
    for _ in range(K):
        for pl in plains:
            od.od2p_iterate(pl, 1)
    e[2].record(s)
    torch.cuda.synchronize()
    tb, tp = e[0].elapsed_time(e[1]) / 1e3, e[1].elapsed_time(e[2]) / 1e3
    same = all(torch.equal(od.od2p_get_state(batch.members[i], k), od.od2p_get_state(plains[i], k))
               for i in range(len(plains)) for k in (od.STATE_U, od.STATE_GAMMA, od.STATE_LAMBDA))
    blaunch = od.ptycho_batch_get_launch(batch)
    for pl in plains:
        pl.close()
    batch.close()
    return {"workload": f"{count} independent reconstructions (images 256-992, probes 32/64/128, "
                        "steps 8-m/2, grids 2x2-8x8, Poisson 1e3-1e5, seed 3)",
            "frames": J, "iterations": K,
            "batched_frame_updates_per_s": round(J * K / tb, 1),
            "plain_frame_updates_per_s": round(J * K / tp, 1),
            "speedup": round(tp / tb, 3),
            "equal_error": ("bitwise identical states (u, Gamma, Lambda) after the same iterations" if same
                            else "states differ"),
            "launches_per_iteration": {"batched": len({g.m for g in geoms}) + 1, "plain": 2 * len(geoms)},
            "batch_launch": {"variant": blaunch[0], "blocks_per_sm": blaunch[1]}}


def measure_workload(od, p, blind: bool, f_host: np.ndarray, dev, K: int, W: int, flush_l2: bool, args,
                     clk=None, stage_iters: int | None = None):
    """Plan, Step 0, launch-shape tuning, W warm-up iterations, then K timed
    graph-replayed iterations (events around each) and stage_iters iterations
    launched stage by stage with events around each stage."""
    import torch

    from paper_2011_00162_gb300 import autotune
    offs = p.offsets()
    J = len(offs)
    geom = _geometry(od, p, offs, blind)
    f_dev = torch.from_numpy(f_host).to(dev)
    w0 = _initial_probe(p, blind)
    plan = od.ptycho_plan(geom, f_dev)
    del f_dev
    od.od2p_init(plan, torch.from_numpy(w0).to(dev))
    # launch shape of the frame update, measured once per workload and cached on
    # disk (tuning restores the plan's state; the candidates give the same iterates)
    tuned = autotune.tune_plan(plan, flush_l2=flush_l2, use_cache=not args.retune) if not args.no_tune else None
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev) if flush_l2 else None
    stream = torch.cuda.current_stream()
    for _ in range(W):
        if flush is not None:
            flush.fill_(1.0)
        od.od2p_iterate(plan, 1)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    Kk = stage_iters if stage_iters is not None else K
    evk = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(Kk)]
    if clk is not None:  # keep the GPU busy while nvidia-smi starts sampling
        t_end = time.perf_counter() + 0.6
        while time.perf_counter() < t_end:
            od.od2p_iterate(plan, 2)
            torch.cuda.synchronize()
        clk.mark_start()
    wall0 = time.perf_counter()
    for k in range(K):
        if flush is not None:
            flush.fill_(float(k))
        ev[k][0].record(stream)
        od.od2p_iterate(plan, 1)  # graph replay of the whole iteration
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall1 = time.perf_counter()
    # per-stage durations for the roofline: the same iteration launched stage by
    # stage, events on the launch stream around each stage
    for k in range(Kk):
        if flush is not None:
            flush.fill_(float(k))
        evk[k][0].record(stream)
        od.od2p_frame_update(plan)
        evk[k][1].record(stream)
        if blind:
            od.probe_update(plan)
        evk[k][2].record(stream)
        od.od2p_subdomain_update(plan)
        evk[k][3].record(stream)
    torch.cuda.synchronize()
    # the frame update alone, replayed from its own CUDA graph as the iteration's
    # graph runs it (no host launch gaps between its kernels): the roofline's time
    g_fu = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    cap.wait_stream(stream)
    with torch.cuda.graph(g_fu, stream=cap):
        od.od2p_frame_update(plan)
    torch.cuda.synchronize()
    evg = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(Kk)]
    for k in range(Kk):
        if flush is not None:
            flush.fill_(float(k))
        evg[k][0].record(stream)
        g_fu.replay()
        evg[k][1].record(stream)
    torch.cuda.synchronize()
    if clk is not None:
        clk.mark_end()
    k1g_ms = [evg[k][0].elapsed_time(evg[k][1]) for k in range(Kk)]
    del g_fu
    step_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(K)]
    k1_ms = [evk[k][0].elapsed_time(evk[k][1]) for k in range(Kk)]
    pu_ms = [evk[k][1].elapsed_time(evk[k][2]) for k in range(Kk)]
    k2_ms = [evk[k][2].elapsed_time(evk[k][3]) for k in range(Kk)]
    rf, re, loss = od.od2p_metrics(plan, loss=True)
    u_true = p.truth()
    snr_db = od.od2p_snr(plan, torch.from_numpy(np.asarray(u_true, np.complex64)).to(dev))
    launch = od.ptycho_plan_get_launch(plan)
    fft_kind = od.ptycho_plan_get_fft(plan)
    out = {"plan": plan, "geom": geom, "offs": offs, "w0": w0, "J": J, "step_ms": step_ms, "k1_ms": k1_ms,
           "k1g_ms": k1g_ms,
           "pu_ms": pu_ms, "k2_ms": k2_ms, "wall_s": wall1 - wall0, "rf": rf, "re": re, "loss": loss,
           "snr_db": snr_db, "launch": launch, "fft_kind": fft_kind, "tuned": tuned,
           "launches_per_iteration": launches_per_iteration(od, plan), "k1_launches": _k1_launches(od, plan),
           "waves": od.ptycho_plan_get_waves(plan)}
    return out


def _k1_name(m: int, launch, fft_kind: int, waves=(0, 1, 1)) -> str:
    if m == 256:
        return ("frame_update256_cluster_kernel<16> (one launch, a 16-CTA cluster per frame)" if launch[0] == 1
                else f"rows_fwd256 / cols256<PROX> / rows_inv256 (three passes per wave of {waves[0]} frames, "
                     f"{waves[1]} chains of waves side by side)")
    if fft_kind:
        return f"frame_update_f4_kernel<{2 - fft_kind}> (16 x 4 transform split, fft kind {fft_kind})"
    return f"frame_update_kernel<{m}, variant {launch[0]}> (two-stage transform split)"


def _traffic_256(variant: int):
    """DRAM bytes per frame of the m = 256 frame update (all of its launches)
    from the committed ncu summary of that variant, when it was taken on the
    current kernel source (else None)."""
    try:
        txt = open(TRAFFIC_FILE_256.format(variant=variant)).read()
    except OSError:
        return None
    src = tr = None
    for line in txt.splitlines():
        if line.startswith("kernel_source_sha256_16:"):
            src = (line.split(":", 1)[1].split() or [""])[0]
        if line.startswith("dram_bytes_per_frame:"):
            tr = (line.split(":", 1)[1].split() or [""])[0]
    h = hashlib.sha256()
    for rel in ("paper_2011_00162_gb300/csrc/fft256_kernels.cu", "paper_2011_00162_gb300/csrc/fft_device.cuh"):
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    if src != h.hexdigest()[:16] or tr is None:
        return None
    try:
        return float(tr)
    except ValueError:
        return None


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2011_00162_gb300 as od
    from paper_2011_00162_gb300 import build as odbuild

    ws, rank, local = _dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        odbuild.build()
    if ws > 1:
        dist.barrier()
    p = _problem()
    f = simulate_intensities(p, seed=7)
    K, W = args.steps, args.warmup
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        r = measure_workload(od, p, True, f, dev, K, W, False, args, clk=clk, stage_iters=min(K, 50))
    if ws > 1:
        dist.barrier()
    J = r["J"]
    total_s = sum(r["step_ms"]) / 1e3
    if ws > 1:
        t = torch.tensor([total_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    value = J * K * ws / total_s
    launch, fft_kind = r["launch"], r["fft_kind"]
    r["plan"].close()
    del r["plan"]
    torch.cuda.empty_cache()

    # ---- end to end through the public API with host buffers (per reconstruction)
    e2e = None
    if not args.no_e2e:
        e2e = e2e_run(od, r["geom"], f, r["w0"], r["offs"], p, dev, ws, tune=not args.no_tune,
                      n_e2e=2 if p.n_iter * statistics.mean(r["step_ms"]) > 300 else 3)
        torch.cuda.empty_cache()

    peak, peak_kind = _peaks()
    alg_bytes = 20.0 * p.m * p.m * J  # f 4 B + Gamma read 8 B + write 8 B per frame pixel
    k1_avg_s = statistics.mean(r["k1g_ms"]) / 1e3  # the frame update replayed from its own graph
    achieved = alg_bytes / k1_avg_s / 1e9
    tpf = _traffic_256(launch[0]) if p.m == 256 else None
    clocks = clk.summary()
    tuned = r["tuned"]
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": W, "ms_per_step": round(statistics.mean(r["step_ms"]), 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded sample, probe and scan; intensities simulated on the host with Poisson noise)",
        "config": {**_config_dict(p, J),
                   "step": "one blind ADMM iteration (Algorithm 3 Steps 1-5, all frames), replayed as a CUDA graph",
                   "l2": "inputs larger than L2 (about 12 GB of frame traffic per iteration against 129 MB)",
                   "parallelism": f"replicas{ws}" if ws > 1 else "single-gpu",
                   "frame_update_ms": round(statistics.mean(r["k1g_ms"]), 5),
                   "frame_update_stage_launched_ms": round(statistics.mean(r["k1_ms"]), 5),
                   "probe_update_ms": round(statistics.mean(r["pu_ms"]), 5),
                   "subdomain_update_ms": round(statistics.mean(r["k2_ms"]), 5),
                   "stage_timing": f"{len(r['k1_ms'])} more iterations launched stage by stage (events around "
                                   "each stage), then the frame update replayed from its own CUDA graph "
                                   f"{len(r['k1g_ms'])} times (frame_update_ms, the roofline's time), after the "
                                   "timed steps",
                   "rf_after": r["rf"], "re_after": r["re"], "loss_after": r["loss"],
                   "snr_db_after": round(r["snr_db"], 3),
                   "launch": {"variant": launch[0], "fft": fft_kind,
                              "tuned": None if tuned is None else
                              {"cached": tuned["cached"], "trials_us": tuned.get("trials")}}},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": None if tpf is None else round(tpf * J, 1),
                     "kernel": _k1_name(p.m, launch, fft_kind, r["waves"]),
                     "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "frame_update_launches": r["k1_launches"]},
        "e2e": e2e,
        "gpu_launches": r["launches_per_iteration"] * K,
        "clocks": clocks,
        "wall_s_timed_region": round(r["wall_s"], 4),
    }
    if not args.no_config2:
        line["config2"] = config2_leg(od, dev, args)
    if not args.no_batched:
        line["batched"] = batched_leg(od, dev, tune=not args.no_tune, retune=args.retune)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, budget_s=args.cpu_budget)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def config2_leg(od, dev, args, K: int = 200, W: int = 5):
    """The 512^2 / 841-frame / 64^2 nonblind workload, L2 flushed before each timed iteration."""
    import torch
    p = _problem2()
    f = simulate_intensities(p, seed=7)
    r = measure_workload(od, p, False, f, dev, K, W, True, args)
    r["plan"].close()
    torch.cuda.empty_cache()
    J = r["J"]
    peak, _ = _peaks()
    k1 = statistics.mean(r["k1g_ms"]) / 1e3
    fft_kind, launch = r["fft_kind"], r["launch"]
    return {"workload": WORKLOAD2, "value": round(J * K / (sum(r["step_ms"]) / 1e3), 1), "unit": UNIT,
            "steps": K, "ms_per_step": round(statistics.mean(r["step_ms"]), 5),
            "frame_update_ms": round(1e3 * k1, 5), "subdomain_update_ms": round(statistics.mean(r["k2_ms"]), 5),
            "frame_update_hbm_frac": round(20.0 * p.m * p.m * J / k1 / 1e9 / peak, 4),
            "kernel": _k1_name(p.m, launch, fft_kind, r["waves"]),
            "l2": "flushed before every timed step (256 MiB write, outside the timed interval)",
            "rf_after": r["rf"], "re_after": r["re"], "snr_db_after": round(r["snr_db"], 3),
            "launch": {"variant": launch[0], "blocks_per_sm": launch[1], "fft": fft_kind}}


# ----------------------------------------------------------------------------- all workloads
def _torus_offsets(p, n=None):
    """A raster over the whole torus of side n (default p.n) with p's step and
    jitter, wrapped modulo the image: the scan of a periodic workload."""
    n = p.n if n is None else n
    offs = np.array([(r, c) for r in range(0, n, p.step) for c in range(0, n, p.step)], np.int32)
    if p.jitter:
        offs = offs + np.random.default_rng(p.seed + 1000).integers(-p.jitter, p.jitter + 1, offs.shape)
    return (offs % n).astype(np.int32)


def _gpu_problem_inputs(od, p, dev, seed: int = 7, periodic: bool = False):
    """Truth, probe, scan and intensities for problem p, the intensities made on
    the GPU (the library's forward operator, torch.poisson at p.peak); periodic:
    a scan over the whole torus and windows that wrap."""
    import torch
    offs = _torus_offsets(p) if periodic else p.offsets()
    u_true, w = p.truth(), p.probe()
    tmp = od.ptycho_plan(od.Geometry(p.n, p.n, p.m, offs, periodic=periodic),
                         torch.ones((len(offs), p.m, p.m), dtype=torch.float32, device=dev))
    fr = od.ptycho_forward(tmp, torch.from_numpy(u_true).to(dev), torch.from_numpy(w).to(dev))
    tmp.close()
    f = fr.abs().square_()
    del fr
    if p.peak is not None:
        gen = torch.Generator(device=dev)
        gen.manual_seed(seed)
        kappa = float(p.peak) / float(f.max())
        f = torch.poisson(f.mul_(kappa), generator=gen).div_(kappa)
    return offs, u_true, w, f.float().contiguous()


def _event_times(fn, K: int, flush):
    """Per-call device times (s) of K calls of fn, the L2 flushed before each."""
    import torch
    s = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for k in range(K):
        flush.fill_(float(k))
        ev[k][0].record(s)
        fn()
        ev[k][1].record(s)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) / 1e3 for a, b in ev]


def _oracle_sample(p, blind, params, budget_s, max_frames, periodic: bool = False):
    """Frame-updates/s of the FP64 oracle on the host cores, on a bounded sample of
    problem p: a square crop holding at most max_frames frames of the same probe,
    step and subdomain grid (periodic: a smaller torus with the same step),
    iterated until budget_s has passed (at least once)."""
    import dataclasses

    import oracle
    from paper_2011_00162_gb300 import synth
    if periodic:
        n = p.n
        while n > 2 * p.m and (n // p.step) ** 2 > max_frames:
            n -= p.step
    else:
        n = p.m + ((p.n - p.m) // p.step) * p.step
        while n > 2 * p.m and len(synth.raster_offsets(n, p.m, p.step)) > max_frames:
            n -= p.step
    grid = max(2, n // (2 * p.m)) if n >= 2 * p.m else 1
    q = dataclasses.replace(p, n=n, sub_rows=min(p.sub_rows, grid), sub_cols=min(p.sub_cols, grid))
    offs = _torus_offsets(q) if periodic else q.offsets()
    u_true, w = q.truth(), q.probe()
    f = synth.poissonize(np.abs(oracle.forward(u_true, w, offs, periodic=periodic)) ** 2, q.peak, 7)
    w0 = synth.gaussian_probe(q.m) if blind else w
    a = oracle.ADMM(f, w0, offs, q.n, q.n, q.sub_rows, q.sub_cols, q.overlap_px, q.eps, params["eta"],
                    params["r"], blind=blind, mu=params.get("mu", 0.0), gamma=params.get("gamma", 0.0),
                    periodic=periodic)
    it = 0
    t0 = time.perf_counter()
    while True:
        a.iterate(1)
        it += 1
        el = time.perf_counter() - t0
        if el > budget_s:
            break
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": round(len(offs) * it / el, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{it} oracle iterations of a {q.n}^2 {'torus' if periodic else 'crop'} ({len(offs)} frames "
                      f"of {q.m}^2, {q.sub_rows}x{q.sub_cols} subdomains), {el:.1f} s"}


def run_configs(args):
    """One JSON line per workload: GPU iteration throughput (L2 flushed per
    iteration), gradient throughput of the ST-AGM loss with exit-wave recompute
    (blind workloads), and the oracle on a bounded sample."""
    import torch

    import paper_2011_00162_gb300 as od
    from paper_2011_00162_gb300 import autotune, synth
    from paper_2011_00162_gb300 import build as odbuild
    odbuild.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    table = [
        ("config1_od2p_64px_m16_169frames_1x2sub_noiseless", synth.small_2sub(), False,
         {"eta": 0.1, "r": 0.05}, 2000),
        ("config2_od2p_512px_m64_841frames_4x4sub_poisson1e4", synth.grid_4x4(), False,
         {"eta": 2.0, "r": 0.5}, 2000),
        ("config4_od2bp_1024px_m128_841frames_4x4sub_poisson1e4", synth.blind_4x4(), True,
         {"eta": 2.0, "r": 0.5, "mu": 1.0, "gamma": 0.1}, 300),
        ("config5_od2bp_4096px_m256_6561frames_8x8sub_poisson1e5", synth.large_blind(), True,
         {"eta": 2.0, "r": 0.5, "mu": 1.0, "gamma": 0.1}, 30),
        # a mixed-radix probe side (80 = 16 x 5) and a periodic scan (windows wrapping around a torus)
        ("mixed_radix_od2p_480px_m80_441frames_3x3sub_poisson1e4",
         synth.Problem("mr80", 480, 80, 20, 2, 3, 3, 16, 1e4, 1), False, {"eta": 2.0, "r": 0.5}, 1000),
        ("periodic_od2bp_512px_m64_1024frames_torus_4x4sub_poisson1e4",
         synth.Problem("per64", 512, 64, 16, 2, 4, 4, 16, 1e4, 1), True,
         {"eta": 2.0, "r": 0.5, "mu": 1.0, "gamma": 0.1}, 1000, True),
    ]
    for name, p, blind, prm, K, *periodic in table:
        periodic = bool(periodic and periodic[0])
        if args.only and args.only not in name:
            continue
        offs, u_true, w, f = _gpu_problem_inputs(od, p, dev, periodic=periodic)
        J = len(offs)
        g = od.Geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px, p.eps, prm["eta"], prm["r"],
                        mu=prm.get("mu", 0.0), gamma=prm.get("gamma", 0.0), blind=blind, periodic=periodic)
        plan = od.ptycho_plan(g, f)
        w0 = torch.from_numpy(synth.gaussian_probe(p.m) if blind else w).to(dev)
        od.od2p_init(plan, w0)
        tuned = autotune.tune_plan(plan, flush_l2=True)
        for _ in range(5):
            flush.fill_(0.0)
            od.od2p_iterate(plan, 1)
        t_it = _event_times(lambda: od.od2p_iterate(plan, 1), K, flush)
        t_k1 = _event_times(lambda: od.od2p_frame_update(plan), max(10, K // 10), flush)
        line = {"workload": name, "frames": J, "image": p.n, "probe": p.m, "blind": blind, "periodic": periodic,
                "subdomains": f"{p.sub_rows}x{p.sub_cols}", "iterations_timed": K,
                "frame_updates_per_s": round(J * K / sum(t_it), 1),
                "ms_per_iteration": round(1e3 * statistics.mean(t_it), 5),
                "frame_update_ms": round(1e3 * statistics.mean(t_k1), 5),
                "hbm_algorithmic_frac_frame_update": round(
                    20.0 * p.m * p.m * J / statistics.mean(t_k1) / 1e9 / _peaks()[0], 4),
                "launch": list(od.ptycho_plan_get_launch(plan)), "tuned_cached": tuned["cached"],
                "l2": "flushed before every timed call"}
        if blind:
            u = od.od2p_merge(plan)
            wcur = od.od2p_get_state(plan, od.STATE_W).reshape(p.m, p.m).contiguous()
            Kg = max(5, K // 3)
            t_g = _event_times(lambda: od.stagm_loss_grad(plan, u, wcur), Kg, flush)
            line["gradient_frames_per_s"] = round(J * Kg / sum(t_g), 1)
            line["ms_per_gradient"] = round(1e3 * statistics.mean(t_g), 5)
            line["gradient"] = "ST-AGM loss + grad_u + grad_w in one call (one pass over the frames, then the gathers)"
            # a loss then a gradient (the autograd pattern): frames recomputed in the
            # second call, or kept by the first (J x m x m complex) and gathered from
            fwd_bwd_re = lambda: (od.stagm_loss_grad(plan, u, wcur, grad_u=False, grad_w=False),
                                  od.stagm_loss_grad(plan, u, wcur))
            fwd_bwd_st = lambda: (od.stagm_loss_grad(plan, u, wcur, grad_u=False, grad_w=False,
                                                     recompute=od.STORE),
                                  od.stagm_loss_grad(plan, u, wcur, recompute=od.FROM_STORE))
            t_re = _event_times(fwd_bwd_re, Kg, flush)
            t_st = _event_times(fwd_bwd_st, Kg, flush)
            line["loss_then_gradient_ms"] = {"recompute": round(1e3 * statistics.mean(t_re), 5),
                                             "stored": round(1e3 * statistics.mean(t_st), 5),
                                             "stored_bytes": J * p.m * p.m * 8}
        rf, re = od.od2p_metrics(plan)
        line["rf_after"], line["re_after"] = rf, re
        line["snr_db_after"] = round(od.od2p_snr(plan, torch.from_numpy(np.asarray(u_true, np.complex64)).to(dev)), 3)
        plan.close()
        del f
        torch.cuda.empty_cache()
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = _oracle_sample(p, blind, prm, budget_s=args.cpu_budget,
                                                  max_frames=200 if p.m >= 128 else 900, periodic=periodic)
        print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- time to solution
def _run_to_rf(od, plan, tol: float, max_it: int, check: int, balance: bool, balance_eta: bool = False):
    """Iterate plan until RF <= tol or max_it.  Without balance the test runs on
    the device after every iteration (od2p_iterate_until); with balance the host
    reads RF every `check` iterations and rebalances r there, and eta too with
    balance_eta (adaptive.decide).
    Returns (iterations, RF, RE, seconds of wall clock, r at the end)."""
    import torch

    from paper_2011_00162_gb300 import adaptive
    eta, r = float(plan.geom.eta), float(plan.geom.r)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if not balance:  # the stopping test on the device after every iteration, inside one graph
        done, rf = od.od2p_iterate_until(plan, tol, max_it)
        sec = time.perf_counter() - t0
        return done, rf, od.od2p_metrics(plan)[1], sec, r
    done, rf, re = 0, float("inf"), float("inf")
    while done < max_it:
        k = min(check, max_it - done)
        if balance_eta:  # Gamma kept before the block's last iteration
            if k > 1:
                od.od2p_iterate(plan, k - 1)
            od.od2p_gamma_snapshot(plan)
            od.od2p_iterate(plan, 1)
        else:
            od.od2p_iterate(plan, k)
        done += k
        rf, re = od.od2p_metrics(plan)  # synchronises
        if rf <= tol:
            break
        r_new = adaptive.decide(r, od.od2p_consensus_residual(plan), r * re) if plan.n_pairs else r
        eta_new = (adaptive.decide(eta, od.od2p_frame_residual(plan), eta * re,
                                   r_min=1.01 * (1.0 - plan.geom.eps) / plan.geom.eps) if balance_eta else eta)
        if r_new != r or eta_new != eta:
            od.od2p_set_penalties(plan, eta_new, r_new)
            eta, r = eta_new, r_new
    torch.cuda.synchronize()
    return done, rf, re, time.perf_counter() - t0, r


def run_table1(args):
    """Table 1's (section 4.2) workload run to its stopping rule on one GPU: a
    512^2 noiseless image, a 64^2 probe, raster step 16 (841 frames), D = 1 ... 10
    stripe subdomains, eps = 0.5, until RF <= 1e-5 (at most 1000 iterations).
    For every D: iterations, RF, RE, SNR and the wall clock from the initial
    state, with fixed (eta, r), with residual balancing of r and of (r, eta), and with Lemma 2.4's
    sufficient (r, eta) from the plan's operator norms; for the D in
    --table1-oracle the FP64 oracle's iteration count on the same data beside it."""
    import dataclasses

    import torch

    import paper_2011_00162_gb300 as od
    from paper_2011_00162_gb300 import adaptive, synth
    from paper_2011_00162_gb300 import build as odbuild
    odbuild.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    eta, r = args.eta, args.r
    base = synth.Problem("table1", 512, 64, 16, 0, 1, 1, 48, None, 1000, eta=eta, r=r)
    offs, u_true, w, f = _gpu_problem_inputs(od, base, dev)
    truth = torch.from_numpy(np.asarray(u_true, np.complex64)).to(dev)
    w_dev = torch.from_numpy(w).to(dev)
    oracle_d = {int(x) for x in args.table1_oracle.split(",") if x.strip()}
    for D in (1, 2, 4, 6, 8, 10):
        p = dataclasses.replace(base, sub_cols=D)
        line = {"workload": f"table1_od2p_512px_m64_841frames_1x{D}stripes_noiseless", "frames": len(offs),
                "subdomains": D, "eta": eta, "r": r, "fft": args.fft, "stop": "RF <= 1e-5 or 1000 iterations",
                "check_every": args.check}
        for mode in ("fixed", "balanced_r", "balanced_r_eta", "in_K"):
            t_plan = time.perf_counter()
            plan = od.ptycho_plan(od.Geometry(p.n, p.n, p.m, offs, 1, D, p.overlap_px, p.eps, eta, r), f)
            od.od2p_init(plan, w_dev)
            if args.fft:
                od.ptycho_plan_set_fft(plan, args.fft)
            torch.cuda.synchronize()
            t_plan = time.perf_counter() - t_plan
            if mode == "in_K":  # Lemma 2.4's sufficient (r, eta) from the plan's operator norms
                r_k, eta_k = adaptive.select_in_K(plan)
                od.od2p_set_penalties(plan, eta_k, r_k)
            od.od2p_iterate(plan, 2)  # both graph parities captured outside the clock ...
            od.od2p_init(plan, w_dev)  # ... then back to the initial state
            it, rf, re, sec, r_end = _run_to_rf(od, plan, 1e-5, 1000, args.check, mode.startswith("balanced"),
                                                mode == "balanced_r_eta")
            rec = {"iterations": it, "rf": rf, "re": re, "snr_db": round(od.od2p_snr(plan, truth), 3),
                   "gpu_seconds": round(sec, 5), "plan_seconds": round(t_plan, 4)}
            if mode.startswith("balanced"):
                rec["r_end"] = r_end
            if mode == "balanced_r_eta":
                rec["eta_end"] = float(plan.geom.eta)
            if mode == "in_K":
                rec["eta"], rec["r"] = eta_k, r_k
            line[mode] = rec
            plan.close()
        if D in oracle_d and not args.no_cpu_baseline:
            import oracle
            fh = f.cpu().numpy().astype(np.float64)
            a = oracle.ADMM(fh, w, offs, p.n, p.n, 1, D, p.overlap_px, p.eps, eta, r)
            t0, it = time.perf_counter(), 0
            while it < 1000:
                a.iterate(args.check)
                it += args.check
                if a.metrics()[0] <= 1e-5:
                    break
            line["oracle_fp64"] = {"iterations": it, "rf": a.metrics()[0], "seconds": round(time.perf_counter() - t0, 2),
                                   "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))}
        print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- profiling case
def run_profile_case(args):
    """A blind m = 256 workload for kernel captures: by default the medium case
    (a few GB on the device, inputs larger than L2) of a 2048^2 image, 256^2
    probe, step 48 +-4 (1444 frames), 4x4 subdomains, Poisson 1e5;
    --profile-n 4096 gives the headline workload (8x8 subdomains).  The frame
    update runs launch variant --profile-variant; five iterations after two of
    warm-up, then one line with the time per iteration."""
    import dataclasses

    import torch

    import paper_2011_00162_gb300 as od
    from paper_2011_00162_gb300 import synth
    from paper_2011_00162_gb300 import build as odbuild
    odbuild.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n = args.profile_n
    grid = 8 if n >= 4096 else 4
    p = dataclasses.replace(synth.large_blind(), name=f"od2bp_{n}px_m256_{grid}x{grid}", n=n, sub_rows=grid,
                            sub_cols=grid)
    offs, u_true, w, f = _gpu_problem_inputs(od, p, dev)
    g = od.Geometry(p.n, p.n, p.m, offs, p.sub_rows, p.sub_cols, p.overlap_px, p.eps, 2.0, 0.5, mu=1.0, gamma=0.1,
                    blind=True)
    plan = od.ptycho_plan(g, f)
    od.od2p_init(plan, torch.from_numpy(synth.gaussian_probe(p.m)).to(dev))
    od.ptycho_plan_set_launch(plan, args.profile_variant, 0)
    od.od2p_iterate(plan, 2)
    flush = torch.empty(1, device=dev)
    t = _event_times(lambda: od.od2p_iterate(plan, 1), 5, flush)
    print(json.dumps({"workload": p.name, "frames": len(offs), "variant": args.profile_variant,
                      "ms_per_iteration": round(1e3 * statistics.mean(t), 4),
                      "rf_after": od.od2p_metrics(plan)[0]}), flush=True)


# ----------------------------------------------------------------------------- ceilings
def run_peaks(args):
    """The FP32 FMA and shared-memory ceilings of this GPU, measured with the
    library's probes (CUDA events, median of 5), beside the frame update's own
    FLOP rate: one JSON line."""
    import torch

    import paper_2011_00162_gb300 as od
    from paper_2011_00162_gb300 import build as odbuild
    odbuild.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    nb = sms * 8
    sink = torch.empty(nb * 256, dtype=torch.float32, device=dev)
    out = {"metric": "ceilings", "sms": sms}
    for kind, iters, per, key, unit in ((od.PROBE_FMA, 20000, 16.0, "fp32_tflops", 1e12),
                                        (od.PROBE_SMEM, 4000, 128.0, "smem_tbs", 1e12)):
        od.ptycho_peak_probe(kind, nb, iters, sink)
        ts = _event_times(lambda: od.ptycho_peak_probe(kind, nb, iters, sink), 5, torch.empty(1, device=dev))
        out[key] = round(nb * 256 * iters * per / statistics.median(ts) / unit, 2)
    # the frame update's FLOPs at 512^2 / 841 frames of 64^2: 2 x 5 m^2 log2(m^2) for the
    # transform pair plus about 50 m^2 for the exit wave, prox, Gamma update and weighting
    m, J = 64, 841
    out["frame_update_flop_per_launch"] = float(J * (10 * m * m * 12 + 50 * m * m))
    print(json.dumps(out), flush=True)


def _oracle_crop(p, max_frames: int = 200):
    """A bounded sample of workload p for the FP64 oracle: the largest square
    crop (side m + k step) whose raster holds at most max_frames frames, with
    the same probe, step, jitter, noise and parameters, and a subdomain grid of
    at most 2 x 2; intensities from simulate_intensities, like the GPU arm's."""
    import dataclasses

    from paper_2011_00162_gb300 import synth
    n = p.m + ((p.n - p.m) // p.step) * p.step
    while n > 2 * p.m and len(synth.raster_offsets(n, p.m, p.step)) > max_frames:
        n -= p.step
    grid = 2 if n >= 2 * p.m else 1
    q = dataclasses.replace(p, n=n, sub_rows=min(p.sub_rows, grid), sub_cols=min(p.sub_cols, grid))
    return q, q.offsets(), simulate_intensities(q, seed=7)


def _oracle_admm(q, offs, f, blind: bool):
    import oracle
    w0 = _initial_probe(q, blind)
    return oracle.ADMM(np.asarray(f, np.float64), w0, offs, q.n, q.n, q.sub_rows, q.sub_cols, q.overlap_px, q.eps,
                       q.eta, q.r, blind=blind, mu=q.mu if blind else 0.0, gamma=q.gamma if blind else 0.0)


def cpu_baseline(p, budget_s: float = 15.0):
    """The FP64 oracle as it stands, on all host cores, on a bounded sample of the
    headline workload (a crop), iterated until budget_s has passed."""
    q, offs, f = _oracle_crop(p)
    a = _oracle_admm(q, offs, f, True)
    n = 0
    t0 = time.perf_counter()
    while True:
        a.iterate(1)
        n += 1
        el = time.perf_counter() - t0
        if el > budget_s or n >= 200:
            break
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"value": round(len(offs) * n / el, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{n} blind oracle iterations of a {q.n}^2 crop of {WORKLOAD} ({len(offs)} frames of "
                     f"{q.m}^2, {q.sub_rows}x{q.sub_cols} subdomains), {el:.1f} s",
           "cpu_model": _cpu_model()}
    one = _one_core_rate()
    if one is not None:
        out["one_core"] = one
    return out


def _cpu_model() -> str:
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20)
        for ln in r.stdout.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def _one_core_rate(steps: int = 2):
    """The reference arm (the oracle) on one host core: a child process with
    OMP_NUM_THREADS=1 timing `steps` iterations of the same workload."""
    env = dict(os.environ, OMP_NUM_THREADS="1", WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--impl", "reference", "--steps", str(steps),
                            "--warmup", "1"], env=env, capture_output=True, text=True, timeout=600)
        line = [ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1]
        d = json.loads(line)
        return {"value": d["value"], "unit": d["unit"], "cores": 1,
                "sample": f"{steps} oracle iterations of the reference arm's crop of {WORKLOAD} on one core"}
    except (OSError, subprocess.SubprocessError, IndexError, ValueError, KeyError):
        return None


def _config_dict(p, J: int) -> dict:
    return {"workload": WORKLOAD, "image": p.n, "probe": p.m, "frames": J, "step_px": p.step,
            "jitter_px": p.jitter, "subdomains": f"{p.sub_rows}x{p.sub_cols}", "overlap_min_px": p.overlap_px,
            "poisson_peak": p.peak, "blind": True, "initial_probe": "Gaussian", "eps": p.eps, "eta": p.eta,
            "r": p.r, "mu": p.mu, "gamma": p.gamma}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, on a bounded sample
    (a crop) of the headline workload, one oracle iteration per step."""
    ws, rank, local = _dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    p = _problem()
    q, offs, f = _oracle_crop(p)
    a = _oracle_admm(q, offs, f, True)
    for _ in range(args.warmup):
        a.iterate(1)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        a.iterate(1)
        ts.append(time.perf_counter() - t0)
    total = sum(ts)
    value = len(offs) * args.steps / total
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"one blind oracle iteration of a {q.n}^2 crop ({len(offs)} frames of {q.m}^2, "
              f"{q.sub_rows}x{q.sub_cols} subdomains) per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded sample, probe and scan; intensities simulated on the host with Poisson noise)",
        "config": _config_dict(p, len(p.offsets())),
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample, "cpu_model": _cpu_model()},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain leg")
    ap.add_argument("--no-config2", action="store_true", help="skip the 512^2 / 841-frame nonblind leg")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shape (no autotuning)")
    ap.add_argument("--retune", action="store_true", help="measure launch shapes even when cached")
    ap.add_argument("--configs", action="store_true",
                    help="measure every workload (one JSON line each) instead of the headline line")
    ap.add_argument("--only", default="", help="with --configs: only workloads whose name contains this")
    ap.add_argument("--profile-case", action="store_true",
                    help="run a medium blind m = 256 workload (2048^2, 1444 frames) for kernel captures")
    ap.add_argument("--profile-n", type=int, default=2048, choices=(2048, 4096),
                    help="with --profile-case: image side (4096: the headline workload)")
    ap.add_argument("--profile-variant", type=int, default=0, choices=(0, 1),
                    help="with --profile-case: launch variant of the m = 256 frame update")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the FP32 FMA and shared-memory ceilings with the library's probes")
    ap.add_argument("--table1", action="store_true",
                    help="run Table 1's workload (section 4.2) (D = 1 ... 10 stripes) to RF <= 1e-5")
    ap.add_argument("--eta", type=float, default=0.1, help="with --table1")
    ap.add_argument("--r", type=float, default=4e3, help="with --table1")
    ap.add_argument("--check", type=int, default=10, help="with --table1: iterations between RF checks")
    ap.add_argument("--fft", type=int, default=0, choices=(0, 1, 2),
                    help="with --table1: transform split of the m = 64 frame update (ptycho_plan_set_fft)")
    ap.add_argument("--table1-oracle", default="1",
                    help="with --table1: comma-separated D for which the FP64 oracle runs the same stopping rule")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
    elif args.peaks:
        run_peaks(args)
    elif args.table1:
        run_table1(args)
    elif args.configs:
        run_configs(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
