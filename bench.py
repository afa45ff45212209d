#!/usr/bin/env python3
"""GGN matvecs/s of the matrix-free LM ptychography solver on one GB300 (or N replicas).

Workload: object 1024x1024, probe 128x128 (defocused disk, radius 40 px), 60x60 jittered
raster (3600 positions, step 15 px: the requested 16 px would carry patches past the
object edge), Poisson counts at 1e3 photons peak, Poisson error metric, complex64 data
with FP64 LM/CG scalars.  Inputs are synthetic and seeded (paper_2103_01767_gb300.synth);
the measurements are simulated with the library's own forward model.

One "step" is one outer iteration of Algorithm 1 through the C-ABI's lm_solve with a fixed
number of CG iterations: linearise (forward + cache + gradient), CG iterations (GGN matvec
+ FP64 dots + vector updates), trial loss, gain ratio and damping update.  `value` counts
the GGN matvecs actually executed (CG iterations plus each solve's initial residual) per
second of device time.  The 472 MB frequency cache streamed by every matvec is larger
than L2, so no L2 flush is needed between steps.

--impl reference times the FP64 CPU oracle (the method's plain restatement) on the host
cores instead, on a bounded sample of positions of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2103_01767_gb300 import synth  # noqa: E402

METRIC = "GGN matvecs/s (1024^2 obj, 3600 pos, 128^2 probe)"   # the headline workload's metric


def metric_for(w):
    """The metric label of workload w (the headline label for the 1024^2 workload)."""
    return f"GGN matvecs/s ({w.n}^2 obj, {w.grid * w.grid} pos, {w.m}^2 probe)"
UNIT = "matvec/s"
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128
HBM_FALLBACK_GBS = 6800.0
PROFILE_FILE = os.path.join(ROOT, "profiles", "ggn_matvec_obj1024_probe128_pos3600.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2103_01767_gb300", "csrc", f)
                  for f in ("team_fft.cuh", "ptycho_device.cuh", "ptycho_kernels.cu", "kernels.h")]


BREAKDOWN_STEPS = 10


def fft_flops(M):
    return 5.0 * M * math.log2(M)


def matvec_flops(K, M):
    """Algorithmic FP32 flops of one GGN matvec: a forward and an inverse M-point 2D FFT per
    position (5 M log2 M each, the usual FFT count) plus 24 flops per pixel of elementwise
    work (probe multiply, frequency stage, conj-probe multiply, scatter add)."""
    return K * (2.0 * fft_flops(M) + 24.0 * M)


def matvec_bytes(K, M, N):
    """Algorithmic DRAM bytes of one GGN matvec: the cache a (8 K M), the vector v and the
    output written and read-modify-written (3 x 8 N), the probe (8 M)."""
    return 8.0 * K * M + 24.0 * N + 8.0 * M


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as fh:
                d = json.load(fh)
            return float(d.get("hbm_gbs") or d.get("hbm_GBs") or HBM_FALLBACK_GBS), "measured"
        except Exception:
            pass
    return HBM_FALLBACK_GBS, "fallback"


def recorded_traffic():
    """dram bytes per matvec launch recorded from an ncu capture of the current kernel
    source (profiles/...md line 'traffic_bytes_per_launch: X kernel_hash: H'); None if the
    kernels changed since."""
    if not os.path.exists(PROFILE_FILE):
        return None
    want = kernel_hash()
    with open(PROFILE_FILE) as fh:
        for line in fh:
            if line.startswith("traffic_bytes_per_launch:"):
                parts = line.split()
                try:
                    val = float(parts[1])
                    hsh = parts[3]
                except (IndexError, ValueError):
                    return None
                return val if hsh == want else None
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for name, flag in zip(names, p[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_config(w, cg_per_step, world):
    _, step_used = synth.raster_positions(w.n, w.m, w.grid, w.step, w.jitter, seed=1)
    return {"workload": w.name, "object": w.n, "probe": w.m, "positions": w.K,
            "problem": "blind (object + probe), PLM-J with Algorithm 2" if w.joint else "object only, LM",
            "raster_step_used": step_used, "loss": "poisson" if w.loss else "amplitude",
            "peak_photons": w.peak, "cg_iters_per_step": cg_per_step, "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2: 8 K M byte cache streamed per matvec"}


def reduce_over_ranks(elapsed_s, count, device):
    """Whole-job figures of N independent replicas (one process per GPU): the slowest
    rank's time and the summed work.  Single-process runs return the inputs unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed_s), float(count)
    t = torch.tensor([float(elapsed_s), float(count)], dtype=torch.float64, device=device)
    tmax, tsum = t.clone(), t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[1])


# ---------------------------------------------------------------------------------------
# CPU legs: the FP64 oracle on a bounded sample of positions
# ---------------------------------------------------------------------------------------
def oracle_sample_problem(w, n_pos, seed=0):
    import oracle
    O_true = synth.to_c64(synth.object_texture(w.n, seed=0))
    P = synth.probe_disk_defocus(w.m, w.radius)
    pos, _ = synth.raster_positions(w.n, w.m, w.grid, w.step, w.jitter, seed=1)
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(pos.shape[0], size=min(n_pos, pos.shape[0]), replace=False))
    pos = pos[idx]
    pb = oracle.Problem((w.n, w.n), P, pos, None, w.loss, 1e-8)
    h = oracle.intensity(pb, O_true)
    if w.peak > 0:
        P = P * np.sqrt(w.peak / h.max())
        pb = oracle.Problem((w.n, w.n), P, pos, None, w.loss, 1e-8)
        h = oracle.intensity(pb, O_true)
        y = synth.poisson_counts(h, seed=2)
    else:
        y = h
    pb.y = np.ascontiguousarray(y, np.float64)
    O = synth.to_c64(synth.flat_object(w.n) * np.mean(np.abs(O_true)))
    v = synth.random_complex((w.n, w.n), seed=3)
    return pb, O, v


def time_oracle_matvec(w, budget_s=15.0):
    """Times oracle.ggn_matvec on a position sample sized for about budget_s seconds.
    Returns (matvecs/s scaled to the full K, seconds, positions, threads)."""
    import oracle
    oracle.build()
    n_try = 16
    pb, O, v = oracle_sample_problem(w, n_try)
    t0 = time.perf_counter()
    oracle.ggn_matvec(pb, O, v, lam=1e-3)
    dt = time.perf_counter() - t0
    n = int(min(w.K, max(n_try, n_try * budget_s / max(dt, 1e-6))))
    pb, O, v = oracle_sample_problem(w, n)
    t0 = time.perf_counter()
    oracle.ggn_matvec(pb, O, v, lam=1e-3)
    dt = time.perf_counter() - t0
    return (n / w.K) / dt, dt, n, oracle.num_threads()


def oracle_op_table(budget_s=1.0):
    """The oracle's forward_loss, J^T w and GGN product at the three single-problem
    workloads, each on a position sample sized for about budget_s seconds and scaled to the
    full K, on all host threads; the GGN product also on one thread."""
    import oracle
    oracle.build()
    threads = oracle.num_threads()
    table = {"threads": threads}
    for w in (synth.SMALL, synth.MEDIUM, synth.LARGE):
        pb, O, v = oracle_sample_problem(w, 4)
        t0 = time.perf_counter()
        oracle.ggn_matvec(pb, O, v, lam=1e-3)
        per = (time.perf_counter() - t0) / 4
        n = int(min(w.K, max(4, budget_s / max(per, 1e-6))))
        pb, O, v = oracle_sample_problem(w, n)
        wts = synth.random_real((n, w.m, w.m), seed=4)
        row = {"positions_timed": n}
        for name, fn in (("forward_loss_s", lambda: oracle.loss(pb, O)),
                         ("jtvp_s", lambda: oracle.jtvp(pb, O, wts)),
                         ("ggn_matvec_s", lambda: oracle.ggn_matvec(pb, O, v, lam=1e-3))):
            t0 = time.perf_counter()
            fn()
            row[name] = (time.perf_counter() - t0) * w.K / n
        n1 = max(2, n // threads)
        pb1, O1, v1 = oracle_sample_problem(w, n1)
        oracle.set_threads(1)
        t0 = time.perf_counter()
        oracle.ggn_matvec(pb1, O1, v1, lam=1e-3)
        row["ggn_matvec_1thread_s"] = (time.perf_counter() - t0) * w.K / n1
        oracle.set_threads(threads)
        table[w.name] = row
    return table


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    threads = oracle.num_threads()
    # size one step at ~4 s of CPU work so warmup+steps finish within a few minutes
    n_try = 8
    pb, O, v = oracle_sample_problem(w, n_try)
    t0 = time.perf_counter()
    oracle.ggn_matvec(pb, O, v, lam=1e-3)
    per_pos = (time.perf_counter() - t0) / n_try
    n = int(min(w.K, max(n_try, 4.0 / max(per_pos, 1e-6))))
    pb, O, v = oracle_sample_problem(w, n)
    for _ in range(args.warmup):
        oracle.ggn_matvec(pb, O, v, lam=1e-3)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.ggn_matvec(pb, O, v, lam=1e-3)
    dt = time.perf_counter() - t0
    value = args.steps * (n / w.K) / dt
    sample = f"{n} of {w.K} positions per step, one FP64 GGN matvec each, scaled by {n}/{w.K}"
    line = {
        "impl": "reference", "metric": metric_for(w), "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w, args.cg_per_step, args.gpus),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------------------
def setup_workload(ptylm, torch, w, dev, stream):
    O_true = torch.from_numpy(synth.object_texture(w.n, seed=0).astype(np.complex64)).to(dev)
    P = torch.from_numpy(synth.probe_disk_defocus(w.m, w.radius).astype(np.complex64)).to(dev)
    pos_np, step_used = synth.raster_positions(w.n, w.m, w.grid, w.step, w.jitter, seed=1)
    pos = torch.from_numpy(pos_np).to(dev)
    y = torch.zeros((pos_np.shape[0], w.m, w.m), dtype=torch.float32, device=dev)
    ctx = ptylm.lm_init(w.n, w.n, w.m, w.m, pos, y, w.loss, 1e-8, joint=int(w.joint), stream=stream)
    ptylm.forward_intensity(ctx, O_true, P, y)
    torch.cuda.synchronize(dev)
    if w.peak > 0:
        P *= math.sqrt(w.peak / float(y.max()))
        ptylm.forward_intensity(ctx, O_true, P, y)
        counts = synth.poisson_counts(y.cpu().numpy(), seed=2).astype(np.float32)
        y.copy_(torch.from_numpy(counts))
    ptylm.ptylm_set_measurements(ctx, y)
    torch.cuda.synchronize(dev)
    O0 = torch.full((w.n, w.n), complex(float(O_true.abs().mean()), 0.0), dtype=torch.complex64, device=dev)
    if w.joint:
        # blind problem: start from the unphased disk with the true probe's integrated intensity
        P0 = torch.from_numpy(synth.probe_disk_defocus(w.m, w.radius, phased=False).astype(np.complex64)).to(dev)
        P0 *= math.sqrt(float((P.abs() ** 2).sum()) / float((P0.abs() ** 2).sum()))
        O0 = torch.full((w.n, w.n), 0.9 + 0.0j, dtype=torch.complex64, device=dev)
        P = P0
    return ctx, O0, P, y, pos, step_used


def measure_fp32_peak(ptylm, dev, stream, launches=10, iters=50000):
    """The library's FFMA loop (ptylm_fp32_peak): every SM's FP32 pipes busy with independent
    FMA chains, 10 timed launches of ~50 ms, median; clocks sampled while it runs."""
    with ClockSampler(dev.index) as clk:
        tflops, ms = ptylm.ptylm_fp32_peak(launches=launches, iters=iters, stream=stream)
    return {"tflops": tflops, "ms_per_launch": ms, "launches": launches, "clocks": clk.summary(),
            "kernel": "k_ffma_loop (2048 threads per SM, 8 independent FMA chains per thread)"}


def matvec_protocol(ptylm, torch, ctx, N, dev, stream, trials=10, min_trial_s=0.2, warmup=10):
    """The GGN product alone, back to back: `warmup` products, then `trials` trials of as many
    products as fill `min_trial_s` each (CUDA events on the context stream around each
    trial), clocks sampled throughout.  The context must hold a linearisation point."""
    v = torch.randn((N,), dtype=torch.complex64, device=dev)
    out = torch.empty_like(v)
    for _ in range(warmup):
        ptylm.ggn_matvec(ctx, v, out, 1e-3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(warmup):
        ptylm.ggn_matvec(ctx, v, out, 1e-3)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    per = e0.elapsed_time(e1) / 1e3 / warmup
    n = max(10, int(math.ceil(min_trial_s / max(per, 1e-6))))
    times = []
    with ClockSampler(dev.index) as clk:
        for _ in range(trials):
            e0.record(stream)
            for _ in range(n):
                ptylm.ggn_matvec(ctx, v, out, 1e-3)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            times.append(e0.elapsed_time(e1) / 1e3 / n)
    med = statistics.median(times)
    return {"trials": trials, "products_per_trial": n, "median_us": 1e6 * med, "min_us": 1e6 * min(times),
            "max_us": 1e6 * max(times), "timed_s": sum(times) * n, "clocks": clk.summary()}


# ---------------------------------------------------------------------------------------
# Comparison and LM time-to-accuracy legs (outside the timed matvec region)
# ---------------------------------------------------------------------------------------
def time_cufft_pair(torch, K, M_side, dev, reps=20):
    """cuFFT (through torch.fft) batched C2C forward + inverse over [K, m, m] complex64: the
    two transforms one GGN matvec needs, without any of its other work.  Comparison only."""
    x = torch.randn((K, M_side, M_side), dtype=torch.complex64, device=dev)
    for _ in range(3):
        y = torch.fft.ifft2(torch.fft.fft2(x, norm="ortho"), norm="ortho")
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        y = torch.fft.ifft2(torch.fft.fft2(x, norm="ortho"), norm="ortho")
    e1.record()
    torch.cuda.synchronize(dev)
    del x, y
    return e0.elapsed_time(e1) * 1e3 / reps


def small_tta_problem():
    """The 128^2 / 32^2 noiseless workload (64 positions, amplitude metric) and its truth."""
    w = synth.SMALL
    O_true = synth.to_c64(synth.object_texture(w.n, seed=0))
    P = synth.to_c64(synth.probe_disk_defocus(w.m, w.radius))
    pos, _ = synth.raster_positions(w.n, w.m, w.grid, w.step, w.jitter, seed=1)
    mask = synth.illumination_mask(w.n, P, pos, 0.1)
    return w, O_true, P, pos, mask


def oracle_time_to_accuracy(target=1e-3):
    """The oracle's plain LM (Algorithm 1, FP64) from the flat start to object error <= target
    on the small noiseless workload, against the ground truth."""
    import oracle
    w, O_true, P, pos, mask = small_tta_problem()
    pb = oracle.Problem((w.n, w.n), P, pos, None, 0, 1e-8)
    pb.y = synth.to_f32(oracle.intensity(pb, O_true))
    t0 = time.perf_counter()
    _, info = oracle.lm_solve(pb, synth.flat_object(w.n), O_ref=O_true, mask=mask, max_outer=100, target_err=target)
    return {"seconds": time.perf_counter() - t0, "outer": int(info["n_outer"]), "err": float(info["err"][-1]),
            "threads": oracle.num_threads()}


def gpu_time_to_accuracy(ptylm, torch, dev, stream, target=1e-3, reps=5, large_ref_outer=200):
    """Wall time of lm_solve (plain LM, data resident after lm_init) from the flat start to the
    first outer iteration with object error <= target, measured on the device each iteration.
      small: 128^2 / 32^2 noiseless, reference = the ground truth (median of reps runs);
      (the large Poisson workload: large_poisson_time_to_accuracy)
    The large workload is timed by large_poisson_time_to_accuracy."""
    out = {}
    w, O_true, P, pos, mask = small_tta_problem()
    c64 = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.complex64)).to(dev)
    posd = torch.from_numpy(pos).to(dev)
    y = torch.zeros((pos.shape[0], w.m, w.m), dtype=torch.float32, device=dev)
    ctx = ptylm.lm_init(w.n, w.n, w.m, w.m, posd, y, 0, 1e-8, stream=stream)
    Od, Pd, maskd = c64(O_true), c64(P), torch.from_numpy(mask.astype(np.uint8)).to(dev)
    ptylm.forward_intensity(ctx, Od, Pd, y)
    ptylm.ptylm_set_measurements(ctx, y)
    O0 = c64(synth.flat_object(w.n))
    runs = []
    for _ in range(reps):
        O = O0.clone()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        _, info = ptylm.lm_solve(ctx, O, Pd, hist_len=100, O_ref=Od, mask=maskd, max_outer=100, target_err=target)
        runs.append((time.perf_counter() - t0, info))
    ptylm.lm_destroy(ctx)
    secs = sorted(r[0] for r in runs)
    info = runs[0][1]
    out["small"] = {"seconds": statistics.median(secs), "outer": int(info["n_outer"]), "cg": int(info["cg_total"]),
                    "err": float(info["err"][-1]), "reference": "ground truth", "runs": reps}

    return out


def converge_with_snapshots(ptylm, torch, dev, ctx, O0, P, max_outer, prefix_s=0.0, **kw):
    """Algorithm 1 from O0 (data resident), one outer iteration per lm_solve_resume call, the
    iterate copied device to device after each (the copies inside the timed region), until the
    damping runs away or max_outer iterations.  Each call linearises afresh (one forward pass
    more per iteration than a single long lm_solve, whose accepted trial doubles as the next
    linearisation), so the times are upper bounds.  Returns (snapshots, seconds after each
    iteration -- prefix_s added --, status, CG iterations)."""
    st = ptylm.new_lm_state(ctx, device=dev)
    O = O0.clone()
    snaps = torch.empty((max_outer,) + tuple(O.shape), dtype=O.dtype, device=dev)
    times, cg = [], 0
    status = ptylm.PTYLM_OK
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for t in range(max_outer):
        status, info = ptylm.lm_solve(ctx, O, P, max_outer=1, state=st, **kw)
        snaps[t].copy_(O)
        torch.cuda.synchronize(dev)
        times.append(time.perf_counter() - t0 + prefix_s)
        cg += info["cg_total"]
        if status == ptylm.PTYLM_ERR_STALLED:
            break
    n = len(times)
    return snaps[:n], np.array(times), status, cg


def snapshot_errors(torch, snaps, ref, mask):
    """Phase-aligned relative object error of every snapshot against ref over the mask (C14;
    reporting only, FP64 on the device after the timed runs)."""
    m = mask.bool()
    b = ref[m].to(torch.complex128)
    nb = torch.linalg.vector_norm(b)
    out = []
    for s in snaps:
        a = s[m].to(torch.complex128)
        c = torch.vdot(a, b)
        out.append(float(torch.linalg.vector_norm(a * (c / c.abs()) - b) / nb))
    return np.array(out)


def blind_errors(torch, snaps, ref, mask, ramp_iterations=3):
    """Object error of every snapshot against ref for the blind problem (C14: solutions are
    unique only up to a complex scale and a linear phase ramp): the ramp a0 + a1 y + a2 x is
    fitted by weighted least squares (weights |o| |r|) to the phase of r conj(o) over the
    mask, the fit repeated so that wrapped phases settle, then the closed-form complex scale
    c = <o, r> / <o, o>; error ||c o - r|| / ||r||.  FP64 on the device, after the runs."""
    m = mask.bool()
    yy, xx = torch.nonzero(m, as_tuple=True)
    A = torch.stack([torch.ones_like(yy), yy, xx], dim=1).to(torch.float64)
    r = ref[m].to(torch.complex128)
    nr = torch.linalg.vector_norm(r)
    out = []
    for s in snaps:
        o = s[m].to(torch.complex128)
        for _ in range(ramp_iterations):
            w = (o.abs() * r.abs()).to(torch.float64)
            ph = torch.angle(r * torch.conj(o))
            Aw = A * w[:, None]   # normal equations of the 3-parameter weighted fit
            coef = torch.linalg.solve(Aw.T @ Aw, Aw.T @ (ph * w))
            o = o * torch.exp(1j * (A @ coef))
        c = torch.vdot(o, r) / torch.vdot(o, o)
        out.append(float(torch.linalg.vector_norm(c * o - r) / nr))
    return np.array(out)


def joint_time_to_accuracy(ptylm, torch, dev, stream, target=1e-3, max_outer=200):
    """Time to object error <= target on the blind 256^2 / 64^2 / 400-position Poisson 1e4
    workload, against the converged plain-LM reconstruction of the joint state z = (O, P)
    (Algorithm 1 with D = I from the flat object and the unphased disk, until the damping
    runs away or max_outer iterations; C15), errors after blind alignment (C14).  Runs: plain
    LM, and PLM-J (D = Dg(G) with Algorithm 2's projections), each also against its own last
    iterate."""
    w = synth.WORKLOADS["obj256_probe64_pos400_poisson_1e4"]
    ctx, O0, P0, y, posd, _ = setup_workload(ptylm, torch, w, dev, stream)
    mask = torch.from_numpy(synth.illumination_mask(w.n, P0.cpu().numpy(), posd.cpu().numpy(), 0.1)
                            .astype(np.uint8)).to(dev)
    runs = {}
    for name, kw in (("LM", dict(scaled=0, projected=0)), ("PLM-J", dict(scaled=1, projected=1))):
        runs[name] = converge_with_snapshots(ptylm, torch, dev, ctx, O0, P0.clone(), max_outer, **kw)
    out = {"workload": "256^2 object / 64^2 probe / 400 positions, joint object and probe, Poisson 1e4 photons peak",
           "target": target, "error": "blind alignment (complex scale and linear phase ramp) on the illuminated pixels",
           "timing": "per-iteration lm_solve_resume calls with a D2D snapshot after each (upper bounds)"}
    O_ref = runs["LM"][0][-1]
    for name, (snaps, times, status, cg) in runs.items():
        e_ref = blind_errors(torch, snaps, O_ref, mask)
        e_own = blind_errors(torch, snaps, snaps[-1], mask)
        s_ref, t_ref = first_below(e_ref, times, target)
        s_own, t_own = first_below(e_own[:-1], times[:-1], target)
        out[name] = {"outer": len(times), "cg": int(cg), "status": int(status), "total_s": float(times[-1]),
                     "vs_plain": {"seconds": s_ref, "outer": t_ref, "err_final": float(e_ref[-1])},
                     "vs_own_limit": {"seconds": s_own, "outer": t_own}}
        del snaps
    out["reference"] = (f"plain LM on z = (O, P) from the flat start, {runs['LM'][0].shape[0]} outer iterations "
                        f"({'the damping ran away' if runs['LM'][2] == ptylm.PTYLM_ERR_STALLED else 'iteration limit'})")
    ptylm.lm_destroy(ctx)
    return out


def first_below(errs, times, target):
    idx = np.flatnonzero(errs <= target)
    return (float(times[idx[0]]), int(idx[0]) + 1) if idx.size else (None, None)


def large_poisson_time_to_accuracy(ptylm, torch, dev, stream, net=None, idx=None, target=1e-3, max_outer=200):
    """Time to object error <= target on the 1024^2 / 128^2 / 3600-position Poisson 1e3
    workload (reading C15).  The reference is the converged plain-LM reconstruction: plain LM
    (Algorithm 1, D = I) from the flat start, run until the damping runs away or max_outer
    iterations.  Every run is timed with per-iteration snapshots; each run's errors are taken
    against the reference ("vs_plain") and against its own last iterate ("vs_own_limit": how
    fast it settles on the point it converges to).  Runs of the same method differ from one
    another at the ~1e-3 level here: the scatter's float reductions round differently from
    run to run, and on this flat, noisy minimum that changes accept / damping decisions."""
    wl = synth.LARGE
    ctx, O0, P, y, posd, _ = setup_workload(ptylm, torch, wl, dev, stream)
    mask = torch.from_numpy(synth.illumination_mask(wl.n, P.cpu().numpy(), posd.cpu().numpy(), 0.1)
                            .astype(np.uint8)).to(dev)
    out = {"workload": "1024^2 / 3600 positions / 128^2 probe, Poisson 1e3 photons peak",
           "target": target,
           "timing": "per-iteration lm_solve_resume calls with a D2D snapshot after each (inside the timed "
                     "region); each call linearises afresh, so the times are upper bounds"}
    runs = {}
    runs["LM"] = converge_with_snapshots(ptylm, torch, dev, ctx, O0, P, max_outer)
    variants = {"PLM": dict(scaled=1), "PLM-S": dict(scaled=1, surrogate_T=20)}
    for name, kw in variants.items():
        runs[name] = converge_with_snapshots(ptylm, torch, dev, ctx, O0, P, max_outer, **kw)
    if net is not None:
        Ol = torch.empty_like(O0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ptylm.learned_init(ctx, net, P, idx, Ol)
        torch.cuda.synchronize(dev)
        init_s = time.perf_counter() - t0
        runs["learned+LM"] = converge_with_snapshots(ptylm, torch, dev, ctx, Ol, P, max_outer, prefix_s=init_s)
        out["learned_init_ms"] = 1e3 * init_s
    O_ref = runs["LM"][0][-1]
    for name, (snaps, times, status, cg) in runs.items():
        e_ref = snapshot_errors(torch, snaps, O_ref, mask)
        e_own = snapshot_errors(torch, snaps, snaps[-1], mask)
        s_ref, t_ref = first_below(e_ref, times, target)
        s_own, t_own = first_below(e_own[:-1], times[:-1], target)
        out[name] = {"outer": len(times), "cg": int(cg), "status": int(status), "total_s": float(times[-1]),
                     "vs_plain": {"seconds": s_ref, "outer": t_ref, "err_final": float(e_ref[-1]),
                                  "err_min": float(e_ref.min())},
                     "vs_own_limit": {"seconds": s_own, "outer": t_own, "err_first": float(e_own[0])},
                     "start_err_vs_plain": float(snapshot_errors(torch, [snaps[0]], O_ref, mask)[0])}
        del snaps
    out["reference"] = (f"plain LM from the flat start, {runs['LM'][0].shape[0]} outer iterations "
                        f"({'the damping ran away' if runs['LM'][2] == ptylm.PTYLM_ERR_STALLED else 'iteration limit'})")
    ptylm.lm_destroy(ctx)
    return out


def learned_vs_plain(ptylm, torch, dev, target=1e-3, pairs=200_000, batch=64, reps=3):
    """Learned initialisation against the flat start (plain LM, Algorithm 1, D = I) on a
    held-out 1024^2 object / 3600 positions / 128^2 probe with noiseless amplitude data:
    train the 6-layer network on `pairs` forward-model pairs cut from 8 other random objects,
    then time, from the data resident on the device, (a) LM from the flat start and (b) the
    stitched network estimate from every 4th raster row and column (225 patterns) followed
    by LM, each to object error <= target against the ground truth (median of reps).
    Returns (results, the trained network, the pattern indices it stitches)."""
    n, m, R = 1024, 128, 40.0
    c64 = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.complex64)).to(dev)
    P = c64(synth.probe_disk_defocus(m, R))
    pool = c64(np.stack([synth.object_texture(n, seed=100 + s) for s in range(8)]))
    widths = (64, 128, 256)
    net = ptylm.net_create(widths, max_batch=batch, seed=1)
    steps = pairs // batch
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    hist = ptylm.net_train(net, pool, 8, n, P, steps=steps, batch=batch, lr=2e-3, seed=5)
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    del pool
    O_true = c64(synth.object_texture(n, seed=0))
    pos_np, _ = synth.raster_positions(n, m, 60, 16, 2, seed=1)
    pos = torch.from_numpy(pos_np).to(dev)
    y = torch.zeros((pos_np.shape[0], m, m), dtype=torch.float32, device=dev)
    ctx = ptylm.lm_init(n, n, m, m, pos, y, 0, 1e-8)
    ptylm.forward_intensity(ctx, O_true, P, y)
    ptylm.ptylm_set_measurements(ctx, y)
    mask = torch.from_numpy(synth.illumination_mask(n, P.cpu().numpy(), pos_np, 0.1).astype(np.uint8)).to(dev)
    idx = torch.from_numpy(np.array([i * 60 + j for i in range(0, 60, 4) for j in range(0, 60, 4)], np.int32)).to(dev)
    flat = torch.full((n, n), complex(float(O_true.abs().mean()), 0.0), dtype=torch.complex64, device=dev)
    O0 = torch.empty_like(flat)

    def run(start_learned):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        if start_learned:
            ptylm.learned_init(ctx, net, P, idx, O0)
            O = O0.clone()
        else:
            O = flat.clone()
        t_init = time.perf_counter() - t0
        _, info = ptylm.lm_solve(ctx, O, P, hist_len=200, O_ref=O_true, mask=mask, max_outer=200, target_err=target)
        return time.perf_counter() - t0, t_init, info

    out = {"network": {"widths": list(widths), "params": net.num_params, "pairs": steps * batch,
                       "train_s": train_s, "loss_first": float(hist[:20].mean()), "loss_last": float(hist[-50:].mean())},
           "workload": "held-out 1024^2 object, 3600 positions, 128^2 probe, noiseless amplitude data, "
                       "reference = ground truth"}
    for name, learned in (("plain", False), ("learned", True)):
        runs = [run(learned) for _ in range(reps + 1)][1:]   # first run warms the path
        secs = sorted(r[0] for r in runs)
        info = runs[0][2]
        err = info["err"][np.isfinite(info["err"])]
        out[name] = {"seconds": statistics.median(secs), "init_ms": 1e3 * statistics.median(r[1] for r in runs),
                     "outer": int(info["n_outer"]), "cg": int(info["cg_total"]),
                     "reached": bool(err.size and err[-1] <= target)}
    ptylm.learned_init(ctx, net, P, idx, O0)
    out["learned"]["start_err"] = _object_error(O0, O_true, mask)
    out["plain"]["start_err"] = _object_error(flat, O_true, mask)
    out["speedup"] = out["plain"]["seconds"] / out["learned"]["seconds"]
    ptylm.lm_destroy(ctx)
    return out, net, idx


def net_layer_flops(widths, m=128):
    """Algorithmic forward flops per pattern of the 6-layer encoder-decoder:
    2 * H_out^2 * C_in * C_out * 9 summed over its 3x3 convolutions."""
    c1, c2, c3 = widths
    ci, co = [2, c1, c2, c3, c2, c1], [c1, c2, c3, c2, c1, 2]
    ho = [m // 2, m // 4, m // 8, m // 4, m // 2, m]
    return [2 * h * h * o * i * 9 for i, o, h in zip(ci, co, ho)]


def net_timing(ptylm, torch, dev, widths=(64, 128, 256), batch_fwd=256, batch_train=64, reps=20):
    """Throughput of the learned initialisation's network on the tensor cores: forward at
    batch_fwd and loss + gradient (forward, input and weight gradients of every layer) at
    batch_train, median wall time of `reps` calls each (device synchronised around every
    call), random inputs.  Algorithmic flops: forward as net_layer_flops, loss + gradient
    three times that."""
    m = 128
    net = ptylm.net_create(widths, max_batch=max(batch_fwd, batch_train), seed=1)
    g = torch.Generator(device="cpu").manual_seed(1)
    X = torch.randn((batch_fwd, 2, m, m), generator=g).to(dev)
    T = torch.randn((batch_train, 2, m, m), generator=g).to(dev)
    mask = torch.from_numpy((np.abs(synth.probe_disk_defocus(m, 40.0)) > 0).astype(np.float32)).to(dev)
    out = torch.empty((batch_fwd, 2, m, m), dtype=torch.float32, device=dev)
    per = float(sum(net_layer_flops(widths, m)))
    res = {"widths": list(widths), "params": net.num_params, "flops_forward_per_pattern": per}
    for name, fn, n, mult in (("forward", lambda: ptylm.net_forward(net, X, out), batch_fwd, 1),
                              ("loss_grad", lambda: ptylm.net_loss_grad(net, X[:batch_train], T, mask),
                               batch_train, 3)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize(dev)
            ts.append(time.perf_counter() - t0)
        ms = 1e3 * statistics.median(ts)
        res[name] = {"batch": n, "ms": ms, "tflops": mult * per * n / (ms * 1e-3) / 1e12}
    net.close()
    return res


def autograd_leg(ptylm, torch, dev, reps=10):
    """The differentiable magnitudes (autograd.far_field_magnitude over the JVP / J^T VP
    kernels) at the 1024^2 / 128^2 / 3600-position geometry, in both memory modes: the unit
    phasor psihat / zeta stored by the forward pass (8 K M bytes; one 2D FFT per position per
    derivative) or the exit waves recomputed in every derivative call (two FFTs, no stored
    array).  Median of `reps` timings (CUDA events) of the forward pass, a reverse-mode J^T w
    (backward of sum w zeta) and a forward-mode J v; and a central-difference check of the
    reverse-mode derivative of L = sum w zeta, w nonzero on the bright pixels of 64 positions."""
    import torch.autograd.forward_ad as fwAD
    from paper_2103_01767_gb300 import autograd as ag
    w_ = synth.LARGE
    P = torch.from_numpy(synth.probe_disk_defocus(w_.m, w_.radius).astype(np.complex64)).to(dev)
    pos_np, _ = synth.raster_positions(w_.n, w_.m, w_.grid, w_.step, w_.jitter, seed=1)
    pos = torch.from_numpy(pos_np).to(dev)
    O = torch.from_numpy(synth.object_texture(w_.n, seed=0).astype(np.complex64)).to(dev)
    K, m = pos_np.shape[0], w_.m
    wts = torch.from_numpy(synth.random_real((K, m, m), seed=5).astype(np.float32)).to(dev)
    v = torch.from_numpy(synth.random_complex((w_.n, w_.n), seed=6).astype(np.complex64)).to(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        ts = []
        for _ in range(reps):
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    out = {"workload": f"{w_.n}^2 object, {m}^2 probe, {K} positions", "reps": reps}
    for mode, budget in (("stored_phasor", 1 << 40), ("recompute_exit_waves", 0)):
        pb = ag.MagnitudeProblem(w_.n, w_.n, m, pos, 1e-8, phasor_budget=budget)
        Od = O.clone().requires_grad_(True)

        def fwd():
            pb._point = None
            return ag.far_field_magnitude(Od, P, pb)

        zeta = fwd()

        def bwd():
            Od.grad = None
            torch.autograd.backward(zeta, wts, retain_graph=True)

        def jvp():
            with fwAD.dual_level():
                fwAD.unpack_dual(ag.far_field_magnitude(fwAD.make_dual(O, v), P, pb)).tangent

        r = {"stores_phasor": pb.stores_phasor, "phasor_bytes": 8 * K * m * m if pb.stores_phasor else 0,
             "forward_ms": timed(fwd), "jtvp_ms": timed(bwd), "jvp_ms": timed(jvp)}
        out[mode] = r
        del pb, zeta, Od
        torch.cuda.empty_cache()
    # central differences of L = sum w zeta (FP64 sums) along v, w on the bright pixels of 64 positions
    pb = ag.MagnitudeProblem(w_.n, w_.n, m, pos, 1e-8, phasor_budget=0)
    with torch.no_grad():
        z0 = ag.far_field_magnitude(O, P, pb)
    sel = torch.zeros(K, dtype=torch.bool, device=dev)
    sel[torch.from_numpy(np.random.default_rng(7).choice(K, 64, replace=False)).to(dev)] = True
    wfd = wts * (z0 > 0.05 * z0.max()).float() * sel[:, None, None].float()
    Od = O.clone().requires_grad_(True)
    L = (ag.far_field_magnitude(Od, P, pb).double() * wfd.double()).sum()
    L.backward()
    dd = float((torch.view_as_real(Od.grad).double() * torch.view_as_real(v).double()).sum())
    eps = 1e-3
    with torch.no_grad():
        Lp = float((ag.far_field_magnitude(O + eps * v, P, pb).double() * wfd.double()).sum())
        Lm = float((ag.far_field_magnitude(O - eps * v, P, pb).double() * wfd.double()).sum())
    fd = (Lp - Lm) / (2 * eps)
    out["central_difference"] = {"positions": 64, "eps": eps, "fd": fd, "adjoint": dd,
                                 "rel_diff": abs(fd - dd) / abs(dd)}
    return out


def _object_error(O, O_ref, mask):
    """Phase-aligned relative error over the mask (host arithmetic on the copies; reporting only)."""
    a = O.cpu().numpy().astype(np.complex128)[mask.cpu().numpy().astype(bool)]
    b = O_ref.cpu().numpy().astype(np.complex128)[mask.cpu().numpy().astype(bool)]
    c = np.vdot(a, b)
    return float(np.linalg.norm(a * (c / abs(c)) - b) / np.linalg.norm(b))


# ---------------------------------------------------------------------------------------
# Batch of 64 independent reconstructions (one persistent launch per operator)
# ---------------------------------------------------------------------------------------
BATCH_METRIC = "batched GGN matvecs/s (64 uneven reconstructions)"
BATCH_UNIT = "problem-matvec/s"


def setup_batch(ptylm, torch, dev, members):
    """Simulate every member's data with the single-problem forward model on the GPU."""
    probs, O0 = [], []
    for mem in members:
        O_true = torch.from_numpy(synth.object_texture(mem.n, seed=mem.seed).astype(np.complex64)).to(dev)
        P = torch.from_numpy(synth.probe_disk_defocus(mem.m, mem.radius).astype(np.complex64)).to(dev)
        pos = torch.from_numpy(synth.batch_positions(mem)).to(dev)
        y = torch.zeros((mem.K, mem.m, mem.m), dtype=torch.float32, device=dev)
        ctx = ptylm.lm_init(mem.n, mem.n, mem.m, mem.m, pos, y, mem.loss, 1e-8)
        ptylm.forward_intensity(ctx, O_true, P, y)
        torch.cuda.synchronize(dev)
        if mem.peak > 0:
            P *= math.sqrt(mem.peak / float(y.max()))
            ptylm.forward_intensity(ctx, O_true, P, y)
            y.copy_(torch.from_numpy(synth.poisson_counts(y.cpu().numpy(), seed=mem.seed + 2).astype(np.float32)))
        ptylm.lm_destroy(ctx)
        probs.append(dict(ny=mem.n, nx=mem.n, m=mem.m, positions=pos, y=y, probe=P, loss=mem.loss, background=1e-8))
        O0.append(torch.full((mem.n * mem.n,), complex(float(O_true.abs().mean()), 0.0), dtype=torch.complex64,
                             device=dev))
    return probs, torch.cat(O0)


def run_batch(args):
    import torch
    from paper_2103_01767_gb300 import build as _build
    _build.build()
    from paper_2103_01767_gb300 import ptylm
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    members = synth.batch_members()
    probs, O0 = setup_batch(ptylm, torch, dev, members)
    bt = ptylm.batch_init(probs, stream=torch.cuda.current_stream(dev))
    ptylm.batch_forward_loss(bt, O0, cache=1)
    choice, tune_ms = ptylm.batch_tune(bt)
    v = torch.randn(bt.total, dtype=torch.complex64, device=dev)
    out = torch.empty_like(v)
    lam = np.full(bt.B, 1e-3)
    for _ in range(args.warmup):
        ptylm.batch_ggn_matvec(bt, v, out, lam)
    torch.cuda.synchronize(dev)
    n0 = ptylm.batch_launches(bt)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        ev0.record()
        for _ in range(args.steps):
            ptylm.batch_ggn_matvec(bt, v, out, lam)
        ev1.record()
        torch.cuda.synchronize(dev)
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = ptylm.batch_launches(bt) - n0
    value = bt.B * args.steps / elapsed
    flops = sum(matvec_flops(m.K, m.m * m.m) for m in members)
    bytes_ = sum(matvec_bytes(m.K, m.m * m.m, m.n * m.n) for m in members)
    clocks = clk.summary()
    fp32 = measure_fp32_peak(ptylm, dev, torch.cuda.current_stream(dev))
    peak_fp32 = fp32["tflops"]
    t_step = elapsed / args.steps
    # e2e: the direction from pinned host memory, the product back to it, every step
    v_h = v.cpu().pin_memory()
    o_h = torch.empty_like(v_h).pin_memory()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(max(1, args.e2e_steps)):
        v.copy_(v_h, non_blocking=True)
        ptylm.batch_ggn_matvec(bt, v, out, lam)
        o_h.copy_(out, non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / max(1, args.e2e_steps)
    # comparison: the same 64 products through 64 single-problem contexts, one after another
    ctxs = []
    for pr, mem in zip(probs, members):
        ctx = ptylm.lm_init(mem.n, mem.n, mem.m, mem.m, pr["positions"], pr["y"], mem.loss, 1e-8)
        ctxs.append(ctx)
    views = bt.views(O0)
    vv, ov = bt.views(v), bt.views(out)
    for c, o, pr in zip(ctxs, views, probs):
        ptylm.forward_loss(c, o, pr["probe"], cache=1)
    for c, a, b in zip(ctxs, vv, ov):
        ptylm.ggn_matvec(c, a, b, 1e-3)
    torch.cuda.synchronize(dev)
    ev0.record()
    reps = 5
    for _ in range(reps):
        for c, a, b in zip(ctxs, vv, ov):
            ptylm.ggn_matvec(c, a, b, 1e-3)
    ev1.record()
    torch.cuda.synchronize(dev)
    seq_s = ev0.elapsed_time(ev1) / 1e3 / reps
    for c in ctxs:
        ptylm.lm_destroy(c)
    # one LM step of all problems (Algorithm 1, 10 CG iterations each, CG under the graph)
    Ob = O0.clone()
    ptylm.batch_lm_solve(bt, Ob, max_outer=1, fixed_cg=10)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    Ob.copy_(O0)
    _, infos = ptylm.batch_lm_solve(bt, Ob, max_outer=1, fixed_cg=10)
    lm_step_s = time.perf_counter() - t0
    # the same step as PLM for every member (D = Dg(G) per problem, Jacobi PCG)
    Ob.copy_(O0)
    ptylm.batch_lm_solve(bt, Ob, max_outer=1, fixed_cg=10, scaled=1)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    Ob.copy_(O0)
    ptylm.batch_lm_solve(bt, Ob, max_outer=1, fixed_cg=10, scaled=1)
    plm_step_s = time.perf_counter() - t0
    line = {
        "metric": BATCH_METRIC, "value": value, "unit": BATCH_UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": synth.BATCH64, "problems": bt.B, "positions": int(sum(m.K for m in members)),
                   "objects": [min(m.n for m in members), max(m.n for m in members)],
                   "probes": sorted({m.m for m in members}), "losses": {"gaussian": sum(m.loss == 0 for m in members),
                                                                         "poisson": sum(m.loss == 1 for m in members)},
                   "step": "one batched GGN product (damping + one persistent launch) over all problems",
                   "parallelism": "replicas1", "l2": "inputs larger than L2: 2.5 GB of caches streamed per step"},
        "roofline": {"bound": "alu", "achieved": flops / t_step / 1e12, "peak": peak_fp32, "unit": "TFLOP/s",
                     "frac": flops / t_step / 1e12 / peak_fp32, "traffic": None, "kernel": "k_batch<matvec>",
                     "peak_kind": "measured in this run: FFMA loop (ptylm_fp32_peak), median of 10 launches",
                     "peak_measured": fp32,
                     "flops_per_launch": flops, "hbm_bytes_per_launch": bytes_},
        "cpu_baseline": None,
        "e2e": {"value": bt.B / e2e_s, "unit": BATCH_UNIT, "h2d_bytes_per_step": 8 * bt.total,
                "d2h_bytes_per_step": 8 * bt.total},
        "clocks": clocks, "gpu_launches": int(launches),
        "schedule": {"chosen": choice, "chosen_desc": ptylm.schedule_desc(choice),
                     "tune_table": [dict(ptylm.schedule_desc(c), schedule=c, ms=t)
                                    for c, t in enumerate(tune_ms) if t > 0],
                     "note": "autotuner over FFT tile (values per thread for the 32^2 / 64^2 problems: "
                             "32 or 16), work-item order and positions per team per item; each entry is "
                             "the mean of 3 batched GGN products"},
        "comparison": {"sequential_single_contexts_ms": 1e3 * seq_s, "batched_ms": 1e3 * t_step,
                       "speedup": seq_s / t_step},
        "lm_step_ms": 1e3 * lm_step_s,
        "plm_step_ms": 1e3 * plm_step_s,
    }
    print(json.dumps(line), flush=True)
    bt.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cg-per-step", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--workload", default=synth.LARGE.name, choices=sorted(synth.WORKLOADS) + [synth.BATCH64])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the cuFFT comparison and the LM time-to-accuracy runs")
    ap.add_argument("--net-timing", action="store_true",
                    help="only time the learned initialisation's network (forward, loss + gradient)")
    args = ap.parse_args()
    if args.net_timing:
        import torch
        from paper_2103_01767_gb300 import build as _build
        _build.build()
        from paper_2103_01767_gb300 import ptylm
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
        torch.cuda.set_device(dev)
        print(json.dumps({"impl": args.impl, "net_timing": net_timing(ptylm, torch, dev)}), flush=True)
        return 0
    if args.workload == synth.BATCH64:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle has no batched form; "
                              "run the single-problem workloads"}), flush=True)
            return 0
        return run_batch(args)
    w = synth.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    # CPU baseline first (before any GPU work, so no forked process ever follows a CUDA call).
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        val, secs, n, threads = time_oracle_matvec(w)
        cpu = {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"one FP64 GGN matvec over {n} of {w.K} positions ({secs:.1f} s), "
                         f"scaled by {n}/{w.K}"}
    oracle_tta = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.no_extras:
        oracle_tta = oracle_time_to_accuracy()
        cpu["ops_full_K"] = oracle_op_table()

    from paper_2103_01767_gb300 import build as _build
    _build.build()
    from paper_2103_01767_gb300 import ptylm

    stream = torch.cuda.current_stream(dev)
    ctx, O0, P, y, pos, step_used = setup_workload(ptylm, torch, w, dev, stream)
    O = O0.clone()
    params = ptylm.default_lm_params(w.loss)
    params.max_outer = 1
    params.fixed_cg = args.cg_per_step
    if w.joint:  # the blind problem needs the scaled, projected variant (PLM-J with Algorithm 2)
        params.scaled = 1
        params.projected = 1
    P_start = P.clone()

    def step(Obuf, Pbuf, Ostart, Pstart=None):
        # every step is the first LM iteration from the same initial guess: constant work
        Obuf.copy_(Ostart)
        if w.joint:
            Pbuf.copy_(P_start if Pstart is None else Pstart)
        st, info = ptylm.lm_solve(ctx, Obuf, Pbuf, params)
        return info["matvecs"]

    for _ in range(args.warmup):
        step(O, P, O0)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    # inside the timed region only the GGN product's launches carry event pairs (roofline)
    mv_kid = ptylm.KERNEL_GGN_MATVEC_JOINT if w.joint else ptylm.KERNEL_GGN_MATVEC
    ptylm.ptylm_profile_select(ctx, [mv_kid])
    # the K timed steps run as (up to) 10 equal trials, each bracketed by its own events
    n_trials = max(1, min(10, args.steps))
    bounds = [round(i * args.steps / n_trials) for i in range(n_trials + 1)]
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(n_trials + 1)]
    matvecs, trial_mv = 0, []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize(dev)
        evs[0].record(stream)
        for i in range(n_trials):
            mv0 = matvecs
            for _ in range(bounds[i + 1] - bounds[i]):
                matvecs += step(O, P, O0)
            evs[i + 1].record(stream)
            trial_mv.append(matvecs - mv0)
        torch.cuda.synchronize(dev)
    elapsed = evs[0].elapsed_time(evs[-1]) / 1e3
    trial_values = [mv / (evs[i].elapsed_time(evs[i + 1]) / 1e3) for i, mv in enumerate(trial_mv)]
    mv_ms, mv_n = ptylm.ptylm_profile_read(ctx, mv_kid)
    _, launches = ptylm.ptylm_profile_read(ctx, -1)
    ptylm.ptylm_profile(ctx, False)
    # per-kernel breakdown from a few more steps with every kernel timed (outside the timed
    # region: the extra event pairs cost ~2 % of a step)
    per_kernel = {}
    ptylm.ptylm_profile(ctx, True)
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    for _ in range(BREAKDOWN_STEPS):
        step(O, P, O0)
    b1.record(stream)
    torch.cuda.synchronize(dev)
    b_elapsed = b0.elapsed_time(b1) / 1e3
    for name, kid in (("forward_cache", ptylm.KERNEL_FORWARD_CACHE_JOINT if w.joint else ptylm.KERNEL_FORWARD_CACHE),
                      ("forward_loss", ptylm.KERNEL_FORWARD_LOSS),
                      ("ggn_matvec", mv_kid),
                      ("cg_iteration", ptylm.KERNEL_CG_ITERATION)):
        ms_k, n_k = ptylm.ptylm_profile_read(ctx, kid)
        if n_k:
            per_kernel[name] = {"avg_us": 1e3 * ms_k / n_k, "launches": int(n_k),
                                "share_of_step": ms_k / (1e3 * b_elapsed) if b_elapsed > 0 else None}
    if per_kernel:
        per_kernel["note"] = (f"{BREAKDOWN_STEPS} steps after the timed region with every kernel timed; "
                              "the timed region times only the GGN product")
    ptylm.ptylm_profile(ctx, False)
    elapsed, total_matvecs = reduce_over_ranks(elapsed, matvecs, dev)
    value = total_matvecs / elapsed
    # outside the timed region: the FP32 peak of this GPU and the GGN product's own protocol
    # (10 trials of back-to-back products, >= 2 s), at the linearisation the last step left
    fp32 = measure_fp32_peak(ptylm, dev, stream)
    protocol = None if w.joint else matvec_protocol(ptylm, torch, ctx, w.n * w.n, dev, stream)

    # End to end through the C-ABI with pinned host buffers: H2D of O and P, D2H of O.
    O0_h = O0.cpu().pin_memory()
    O_h = O0_h.clone().pin_memory()
    P0_h = P_start.cpu().pin_memory()
    P_h = P0_h.clone().pin_memory()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e2e_mv = 0
    for _ in range(args.e2e_steps):
        e2e_mv += step(O_h, P_h, O0_h, P0_h)
    e2e_s = time.perf_counter() - t0
    e2e_s, e2e_mv = reduce_over_ranks(e2e_s, e2e_mv, dev)
    N, M, K = w.n * w.n, w.m * w.m, int(pos.shape[0])

    clocks = clk.summary()
    comparison, tta, autograd = None, None, None
    if rank == 0 and not args.no_extras:
        cufft_us = time_cufft_pair(torch, K, w.m, dev)
        comparison = {"cufft_fwd_inv_us": cufft_us, "matvec_us": 1e6 * (mv_ms / 1e3) / max(mv_n, 1),
                      "note": "cuFFT batched C2C forward + inverse over the same [K, m, m] complex64 "
                              "(torch.fft, comparison only); the matvec adds gather, probe multiplies, "
                              "the frequency stage and the overlap scatter-add"}
        tta = gpu_time_to_accuracy(ptylm, torch, dev, stream)
        if oracle_tta is not None:
            tta["small"]["oracle"] = oracle_tta
        tta["learned_vs_plain"], net, idx = learned_vs_plain(ptylm, torch, dev)
        tta["learned_vs_plain"]["network"]["timing"] = net_timing(ptylm, torch, dev)
        tta["large"] = large_poisson_time_to_accuracy(ptylm, torch, dev, stream, net, idx)
        tta["joint"] = joint_time_to_accuracy(ptylm, torch, dev, stream)
        net.close()
        autograd = autograd_leg(ptylm, torch, dev)
    avg_mv_s = (mv_ms / 1e3) / max(mv_n, 1)
    flops = matvec_flops(K, M)
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_derived = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    peak_fp32 = fp32["tflops"]
    achieved = flops / avg_mv_s / 1e12
    hbm_peak, hbm_kind = measured_peaks()
    hbm_achieved = matvec_bytes(K, M, N) / avg_mv_s / 1e9

    if rank == 0:
        line = {
            "metric": metric_for(w), "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(w, args.cg_per_step, world),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
                         "frac": achieved / peak_fp32, "traffic": recorded_traffic(),
                         "kernel": f"k_ggn_matvec<{int(math.log2(w.m))}{', joint' if w.joint else ''}>",
                         "avg_launch_us": avg_mv_s * 1e6,
                         "launches": mv_n, "flops_per_launch": flops,
                         "peak_kind": "measured in this run: FFMA loop (ptylm_fp32_peak), median of 10 launches",
                         "peak_measured": fp32,
                         "peak_derived": peak_derived,
                         "frac_of_derived": achieved / peak_derived,
                         "peak_basis_derived": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz",
                         "hbm": {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                                 "frac": hbm_achieved / hbm_peak, "peak_kind": hbm_kind,
                                 "bytes_per_launch": matvec_bytes(K, M, N)}},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_mv / e2e_s if e2e_s > 0 else 0.0, "unit": UNIT, "h2d_bytes_per_step": 8 * N + 8 * M,
                    "d2h_bytes_per_step": 8 * N},
            "clocks": clocks,
            "gpu_launches": int(launches),
            "trials": {"n": n_trials, "steps_per_trial": [bounds[i + 1] - bounds[i] for i in range(n_trials)],
                       "values": trial_values, "median": statistics.median(trial_values)},
            "matvec_protocol": protocol,
            "kernels": per_kernel,
            "comparison": comparison,
            "time_to_accuracy": tta,
            "autograd": autograd,
        }
        print(json.dumps(line), flush=True)
    ptylm.lm_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
