#!/usr/bin/env python
"""Benchmark of the MADmap PCG map-making solve on GB300.

Headline workload (default): the all-sky IQU mixed-precision problem, the
largest configuration that fits one GPU: 32 detectors x 2^24 samples
(5.4e8) of a ring scan at 180 Hz on a HEALPix N_side = 512 RING grid,
pointing periods of 40-60 min as stationary intervals, one noise filter
(sigma = 1, f_knee = 0.03 Hz, alpha = 1.7) of 2^15 lags; seeded synthetic data
generated on the GPU.  `--workload config2` runs the same measurement on the
IQU flat-sky problem (4 detectors x 2^22 samples, 512 x 512 pixels).

A step is one complete solve: right-hand side A^T N^-1 d (double-float),
float32 PCG iterations inside float64 iterative refinement, and the
double-float residuals, run to the loosest stopping tolerance whose map is
within 1e-6 (relative RMS per Stokes map) of the reference map.  The reference
map is the FP64 oracle's own PCG solve to relative residual 1e-12 where the
oracle can afford it (config 2, computed on the host before the timed
region); at the all-sky size, whose oracle solve would take hours on the
host, it is the float64 GPU solve to relative residual 1e-11 (the float64
operator and solve are checked against the oracle by the tests, at this size
on sampled rows).  The same time to 1e-6 map error is measured for the plain
float64 GPU solve.  The metric is samples x PCG iterations per second.

--impl reference times the FP64 CPU oracle on bounded samples of the same
workload (one detector's share, one oracle PCG iteration per step, one
process per host core).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

HEADLINE = {
    "config3": ("IQU all-sky mixed precision: 32 det x 2^24 samples (5.4e8) at 180 Hz, ring scan 1 rpm, 85 deg "
                "opening, HEALPix Nside=512 RING, pointing periods 40-60 min, f_knee=0.03 Hz, alpha=1.7, "
                "n_c = 2^15 lags"),
    "config2": ("IQU mixed precision: 4 det x 2^22 samples, 512x512 grid (786,432 unknowns), HWP 22.5 deg/sweep, "
                "intervals 2^16-2^20, n_c = 2^14 lags"),
}
METRIC = "samples x PCG iters/s (time to 1e-6 map error, mixed vs FP64 on the same GPU)"
UNIT = "samples*iters/s"
MAP_TARGET = 1e-6
# stopping tolerances tried, loose to tight (the map error falls as the tolerance tightens)
TOLS = [1e-4, 5e-5, 2e-5, 1e-5, 5e-6, 2e-6, 1e-6, 5e-7, 2e-7, 1e-7, 5e-8, 2e-8, 1e-8, 5e-9, 2e-9, 1e-9,
        5e-10, 1e-10]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-iters", type=int, default=3, help="oracle PCG iterations in the CPU baseline sample")
    ap.add_argument("--cpu-procs", type=int, default=0, help="oracle processes of the all-core CPU baseline "
                                                             "(0 = one per host core, at most 16)")
    ap.add_argument("--workload", default="config3",
                    choices=["config3", "config2", "config1", "config4", "config5", "config2-boresight",
                             "config2-destripe", "config2-multires", "config2-checkpoint"],
                    help="config3 (default) and config2 print the headline measurement; the others print "
                         "secondary measurements")
    ap.add_argument("--profile-step", type=float, default=0.0, metavar="TOL",
                    help="profiling runs: skip the reference map and tolerance search and run exactly one "
                         "mixed-precision solve at this stopping tolerance")
    ap.add_argument("--profile-graph", type=int, default=2, choices=[0, 1, 2],
                    help="iteration driver of the --profile-step solve: 2 device-side graph loop (as timed), "
                         "0 direct launches (every kernel visible to a profiler)")
    ap.add_argument("--fft-len", type=int, default=0, help="override the plan's FFT length (0 = plan's choice)")
    ap.add_argument("--tpc", type=int, default=0, help="override the plan's tiles per launch chunk (0 = plan's choice)")
    ap.add_argument("--det", type=int, default=32,
                    help="detectors of the all-sky workload (profiling captures of a smaller case with the same "
                         "FFT length and kernels; the headline uses all 32)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="plan with the cost model's FFT length instead of the measuring autotuner")
    ap.add_argument("--scatter-runs", type=int, default=0, choices=[-1, 0, 1],
                    help="the operator scatter's run sums: 0 the plan's rule or the autotuner, 1 on, -1 off")
    ap.add_argument("--fft-split", type=int, default=0, choices=[0, 1],
                    help="1: FFT columns half the default length (with --no-autotune; the autotuner times both)")
    ap.add_argument("--inner-tol", type=float, default=1e-4,
                    help="inner float32 tolerance of the --profile-step solve")
    ap.add_argument("--operator-only", type=int, default=0, metavar="R",
                    help="only build the plan and time R float32 operator applications (profiling runs)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed
def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v, device):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, v, device):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers
def stokes_err(m, ref, keep):
    import numpy as np
    out = []
    for s in range(ref.shape[1]):
        a, b = m[keep, s], ref[keep, s]
        out.append(float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)))
    return max(out), out


def operator_source_hash():
    """SHA-256 of the operator's code (comments and blank lines removed, so a comment
    edit does not orphan the committed traffic counters)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("operator_kernels.cuh", "internal.cuh"):
        src = open(os.path.join(ROOT, "paper_0906_1775_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        code = "\n".join(ln.rstrip() for ln in src.splitlines() if ln.strip())
        h.update(code.encode())
    return h.hexdigest()


def lib_lags(p):
    import numpy as np
    import paper_0906_1775_gb300 as mm
    return np.stack([mm.noise_filter(p.n_lags, p.fs, *p.noise_params[k]) for k in range(p.n_filters)])


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ----------------------------------------------------------------------------- CPU oracle
# The FP64 oracle, as it stands, timed on the host: one worker process per
# core (spawned, so no process is forked from one that holds a CUDA context),
# each single-threaded, each running the oracle on its own copy of a bounded
# sample of the workload (one detector's share of the samples).
_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _oracle_worker(job):
    """Worker: build the oracle System over the sample, then either `iters` PCG
    iterations in one run (mode "solve") or `warmup` + `steps` single iterations
    (mode "steps").  Returns (n_samples, iterations, wall seconds, per-step seconds)."""
    import numpy as np
    from multiprocessing import shared_memory

    from oracle.noise import filter_lags
    from oracle.solver import System
    shm = shared_memory.SharedMemory(name=job["shm"])
    try:
        n = job["n"]
        raw = np.ndarray((3, n), dtype=np.int32, buffer=shm.buf)
        pix = raw[0].copy()
        psi = raw[1].view(np.float32).copy()
        d = raw[2].view(np.float32).copy()
    finally:
        shm.close()
    off = np.asarray(job["offsets"], dtype=np.int64)
    filt = np.asarray(job["filter"], dtype=np.int64)
    lags = np.stack([filter_lags(job["n_lags"], job["fs"], *prm) for prm in job["noise"]])
    S = System(pix, psi, job["n_pix"], 3, off, filt, lags)
    b = S.rhs(d)
    if job["mode"] == "solve":
        t0 = time.perf_counter()
        _, info = S.pcg(b, rel_tol=0.0, max_iter=job["iters"])
        return n, max(info["iters"], 1), time.perf_counter() - t0, []
    for _ in range(job["warmup"]):
        S.pcg(b, rel_tol=0.0, max_iter=1)
    times = []
    for _ in range(job["steps"]):
        t0 = time.perf_counter()
        S.pcg(b, rel_tol=0.0, max_iter=1)
        times.append(time.perf_counter() - t0)
    return n, job["steps"], sum(times), times


def run_oracle_workers(sample, n_proc, mode, iters=3, warmup=0, steps=1):
    """Runs n_proc spawned oracle workers on one sample; each worker is one
    single-threaded process.  sample: dict(pix, psi, d, offsets, filter, noise,
    n_lags, fs, n_pix) of host arrays."""
    import multiprocessing as mp
    from multiprocessing import shared_memory

    import numpy as np
    n = int(sample["pix"].shape[0])
    shm = shared_memory.SharedMemory(create=True, size=max(1, 12 * n))
    try:
        raw = np.ndarray((3, n), dtype=np.int32, buffer=shm.buf)
        raw[0] = sample["pix"]
        raw[1] = np.asarray(sample["psi"], dtype=np.float32).view(np.int32)
        raw[2] = np.asarray(sample["d"], dtype=np.float32).view(np.int32)
        job = {"shm": shm.name, "n": n, "offsets": [int(x) for x in sample["offsets"]],
               "filter": [int(x) for x in sample["filter"]], "noise": [list(map(float, r)) for r in sample["noise"]],
               "n_lags": int(sample["n_lags"]), "fs": float(sample["fs"]), "n_pix": int(sample["n_pix"]),
               "mode": mode, "iters": iters, "warmup": warmup, "steps": steps}
        saved = {k: os.environ.get(k) for k in _THREAD_VARS}
        for k in _THREAD_VARS:
            os.environ[k] = "1"
        try:
            ctx = mp.get_context("spawn")
            with ctx.Pool(n_proc) as pool:
                res = pool.map(_oracle_worker, [job] * n_proc)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    finally:
        shm.close()
        shm.unlink()
    return res


def cpu_baseline(sample, iters, n_proc, what):
    """The oracle's samples x iterations / s on one core and on n_proc cores."""
    one = run_oracle_workers(sample, 1, "solve", iters=iters)[0]
    v1 = one[0] * one[1] / one[2]
    out = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{what}: {one[1]} FP64 oracle PCG iterations over its {one[0]} samples in one "
                     f"single-threaded process ({one[2]:.1f} s)"}
    if n_proc > 1:
        res = run_oracle_workers(sample, n_proc, "solve", iters=iters)
        wall = max(r[2] for r in res)
        v = sum(r[0] * r[1] for r in res) / wall
        out = {"value": v, "unit": UNIT, "cores": n_proc, "kind": "oracle",
               "sample": f"{what}: {n_proc} single-threaded processes, one per host core, each running "
                         f"{res[0][1]} FP64 oracle PCG iterations over its own copy of the {res[0][0]} samples "
                         f"(slowest {wall:.1f} s)",
               "single_core": {"value": v1, "cores": 1, "wall_s": one[2]}}
    return out


def cpu_oracle_rate(p, iters):
    """FP64 oracle in this process: samples x PCG iterations / s over `iters` iterations."""
    import numpy as np

    from oracle.noise import filter_lags
    from oracle.solver import System
    lags = np.stack([filter_lags(p.n_lags, p.fs, *p.noise_params[k]) for k in range(p.n_filters)])
    S = System(p.pix, p.psi, p.n_pix, p.n_stokes, p.interval_offsets, p.interval_filter, lags)
    b = S.rhs(p.d[0])
    t0, c0 = time.perf_counter(), time.process_time()
    _, info = S.pcg(b, rel_tol=0.0, max_iter=iters)
    wall, cpu = time.perf_counter() - t0, time.process_time() - c0
    its = max(info["iters"], 1)
    return p.n_samples * its / wall, wall, its, max(1, round(cpu / wall))


def detector_sample(p, det, pix, psi, d):
    """Host copy of detector `det`'s share of a problem (its samples and intervals)."""
    import numpy as np
    idx = np.flatnonzero(np.asarray(p.interval_det) == det)
    off = np.asarray(p.interval_offsets, dtype=np.int64)
    lo, hi = int(off[idx[0]]), int(off[idx[-1] + 1])

    def host(a):
        return a[lo:hi].cpu().numpy() if hasattr(a, "cpu") else np.asarray(a[lo:hi])

    return {"pix": host(pix), "psi": host(psi), "d": host(d), "offsets": np.concatenate([[0], off[idx + 1] - lo]),
            "filter": np.zeros(idx.size, dtype=np.int64) + np.asarray(p.interval_filter)[idx],
            "noise": np.asarray(p.noise_params), "n_lags": p.n_lags, "fs": p.fs, "n_pix": p.n_pix}


# ----------------------------------------------------------------------------- reference arm
def reference_sample(workload):
    """Bounded sample of a headline workload for the host oracle: detector 0's share."""
    import numpy as np
    if workload == "config2":
        from synth import make_config
        p = make_config(2)
        return detector_sample(p, 0, p.pix, p.psi, p.d[0]), "detector 0 of the IQU flat-sky workload"
    from synth.allsky import make_allsky_problem
    p = make_allsky_problem(scale=0, n_det=1, seed=3000)
    s = detector_sample(p, 0, p.pix, p.psi, p.d[0])
    s["noise"] = np.asarray(p.noise_params)
    return s, "one detector (2^24 samples, 31 pointing periods) of the all-sky workload, generated on the host"


def run_reference(args, world, rank):
    if rank != 0:
        return
    workload = args.workload if args.workload in HEADLINE else "config3"
    sample, what = reference_sample(workload)
    n_proc = args.cpu_procs or min(16, host_cores())
    res = run_oracle_workers(sample, n_proc, "steps", warmup=args.warmup, steps=args.steps)
    wall = max(r[2] for r in res)
    value = sum(r[0] * r[1] for r in res) / wall
    ms_step = 1e3 * max(statistics.mean(r[3]) for r in res)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": HEADLINE[workload], "l2_flush": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n_proc, "kind": "oracle",
                             "sample": f"{what}: per step, one FP64 oracle PCG iteration (H application + CG "
                                       f"update) in each of {n_proc} single-threaded processes, one per host core"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- secondary workloads
def _timed(fn, reps):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = None
    for _ in range(reps):
        out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def run_secondary(args):
    import numpy as np
    import torch

    import paper_0906_1775_gb300 as mm
    from synth import make_config
    from synth.flat import device_timestreams
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    mm.load()
    steps, warm = max(1, args.steps), max(1, args.warmup)
    line = {"workload": args.workload, "unit": UNIT}
    if args.workload == "config1":
        p = make_config(1)
        plan = mm.Plan(torch.from_numpy(p.pix).to(dev), None, p.n_pix, p.interval_offsets, p.interval_filter,
                       lib_lags(p))
        d = torch.from_numpy(p.d[0]).to(dev)
        for prec in ("fp64", "mixed"):
            fn = lambda: plan.solve(d, precision=prec, rel_tol=1e-8, max_iter=500)  # noqa: E731
            for _ in range(warm):
                fn()
            ms, (m, info) = _timed(fn, steps)
            line[prec] = {"ms_per_solve": ms, "iters": info["iters"], "rel_res": info["best_rel_res"],
                          "value": p.n_samples * info["iters"] / (ms / 1e3)}
        v, wall, its, cores = cpu_oracle_rate(p, 13)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"full FP64 oracle solve to 1e-8 ({its} iterations, {wall:.2f} s)"}
        line["workload_desc"] = "T-only FP64, 1 det, 2^18 samples, 64x64, n_c=2^12, rel. residual 1e-8"
    elif args.workload == "config4":
        n_rhs = 64
        p = make_config(4, n_rhs=0)
        d = device_timestreams(p, n_rhs, seed=4000, device=dev)
        plan = mm.Plan(torch.from_numpy(p.pix).to(dev), None, p.n_pix, p.interval_offsets, p.interval_filter,
                       lib_lags(p))
        kw = dict(precision="mixed", rel_tol=1e-8, max_iter=500, max_outer=10)
        plan.solve_batched(d[:2].contiguous(), **kw)
        ms_b, (mb, infos) = _timed(lambda: plan.solve_batched(d, **kw), 1)
        rows = [d[r].contiguous() for r in range(n_rhs)]
        plan.solve(rows[0], **kw)
        torch.cuda.synchronize()
        ms_s, its_s = 0.0, 0
        for r in range(n_rhs):
            t, (_, info) = _timed(lambda: plan.solve(rows[r], **kw), 1)
            ms_s += t
            its_s += info["iters"]
        its_b = sum(i["iters"] for i in infos)
        line.update({"n_rhs": n_rhs, "n_samples": p.n_samples, "fft_len": plan.stats["fft_len"],
                     "batched": {"ms": ms_b, "iters_total": its_b, "value": p.n_samples * its_b / (ms_b / 1e3)},
                     "sequential": {"ms": ms_s, "iters_total": its_s, "value": p.n_samples * its_s / (ms_s / 1e3)},
                     "speedup_batched_vs_sequential": ms_s / ms_b,
                     "workload_desc": "T, 64 RHS over one pointing, 500 intervals 2^12-2^20, n_c=2^12, mixed to 1e-8"})
    elif args.workload == "config2-destripe":
        # destriping run (white noise, one offset per 6000-sample baseline) over the
        # IQU workload's pointing, next to the full noise model's operator
        from synth.extended import add_extra_signal, baseline_index
        p = make_config(2)
        idx, n_extra = baseline_index(p.n_samples // 4, 4, 6000)
        d_host = add_extra_signal(p.d[0], idx, np.random.default_rng(7).normal(0.0, 1.0, n_extra))
        pix, psi = torch.from_numpy(p.pix).to(dev), torch.from_numpy(p.psi).to(dev)
        eidx = torch.from_numpy(idx).to(dev)
        white = np.ones((p.n_filters, 1))
        plan = mm.Plan(pix, psi, p.n_pix, p.interval_offsets, p.interval_filter, white, extra_index=eidx,
                       n_extra=n_extra)
        if args.operator_only:      # a short run of the diagonal pass alone (for ncu)
            ms, n = plan.time_operator("fp32", reps=args.operator_only)
            print(json.dumps({"operator_only": "config2-destripe", "fp32_ms": [float(x) for x in ms],
                              "launches": [int(x) for x in n]}), flush=True)
            plan.close()
            return
        d = torch.from_numpy(d_host).to(dev)
        ops = {}
        for prec in ("fp32", "df64", "fp64"):
            ms, n = plan.time_operator(prec, reps=20 if prec == "fp32" else 5)
            ops[prec + "_ms"] = float(ms[3])
        n_rows = plan.n_obs
        b_alg = p.n_samples * (8 + 4) + 2 * n_rows * 4 * 4      # (pixel, angle) + extra index; map read + written
        hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0)) \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
        ref, rinfo = plan.solve(d, precision="fp64", rel_tol=1e-11, max_iter=5000)
        ref_h = ref.cpu().numpy()
        keep = np.ones(n_rows, dtype=bool)
        keep[:n_rows - n_extra] = ~plan.observed()[1].cpu().numpy().astype(bool)
        solves = {}
        for prec, kw in (("mixed", dict(max_outer=30)), ("fp64", {})):
            fn = lambda: plan.solve(d, precision=prec, rel_tol=1e-7, max_iter=5000, **kw)  # noqa: E731
            fn()
            ms_t, (m, info) = _timed(fn, steps)
            err, per = stokes_err(m.cpu().numpy(), ref_h, keep)
            solves[prec] = {"ms": ms_t, "iters": info["iters"], "map_err": err,
                            "value": p.n_samples * info["iters"] / (ms_t / 1e3)}
        full = mm.Plan(pix, psi, p.n_pix, p.interval_offsets, p.interval_filter, lib_lags(p), extra_index=eidx,
                       n_extra=n_extra)
        full_ms, _ = full.time_operator("fp32", reps=10)
        full.close()
        # the same destriping pass with the 32-parameter half-wave-plate model, one group per detector
        from synth.extended import hwp_inputs
        ang, tau, _, _ = hwp_inputs(p.interval_offsets, p.fs, 2.0, np.random.default_rng(8))
        hplan = mm.Plan(pix, psi, p.n_pix, p.interval_offsets, p.interval_filter, white, extra_index=eidx,
                        n_extra=n_extra, hwp=(torch.from_numpy(ang).to(dev), torch.from_numpy(tau).to(dev),
                                              p.interval_det, 4))
        hwp_ms, _ = hplan.time_operator("fp32", reps=10)
        hplan.close()
        line.update({"n_samples": p.n_samples, "n_extra": n_extra, "rows": n_rows,
                     "operator_diag": ops, "alg_bytes": int(b_alg),
                     "hbm": {"achieved_gbs": b_alg / (ops["fp32_ms"] * 1e-3) / 1e9, "peak_gbs": hbm,
                             "frac": b_alg / (ops["fp32_ms"] * 1e-3) / 1e9 / hbm},
                     "operator_full_noise_fp32_ms": float(full_ms[3]),
                     "operator_diag_with_hwp_fp32_ms": float(hwp_ms[3]),
                     "speedup_destripe_vs_full_noise_operator": float(full_ms[3]) / ops["fp32_ms"],
                     "solve_to_rel_res_1e-7": solves,
                     "reference": f"FP64 GPU solve to rel. residual 1e-11 ({rinfo['iters']} iterations)",
                     "workload_desc": "IQU destriping: the IQU workload's pointing (4 det x 2^22, 512x512), white "
                                      "noise, offsets on 6000-sample baselines (one reference baseline)"})
        plan.close()
    elif args.workload == "config2-multires":
        # the IQU workload with Q and U on a 256 x 256 grid (2 x 2 intensity pixels each)
        from synth.flat import log_uniform_intervals
        from synth import make_flat_problem

        def ivls(rng, n):
            return log_uniform_intervals(n, 1 << 16, 1 << 20, rng)

        def nz(rng, nd):
            return np.stack([np.ones(nd), rng.uniform(0.05, 0.2, nd), rng.uniform(1.0, 2.0, nd)], 1)

        p = make_flat_problem("config2-multires", 2000, 512, 4, 1 << 22, 3, 1 << 14,
                              det_angles_deg=[0.0, 45.0, 90.0, 135.0], hwp_step_deg=22.5, interval_lengths=ivls,
                              noise=nz, pol_factor=2)
        pix, psi = torch.from_numpy(p.pix).to(dev), torch.from_numpy(p.psi).to(dev)
        d = torch.from_numpy(p.d[0]).to(dev)
        res = {}
        for name, kw in (("single_resolution", {}),
                         ("multi_resolution", dict(pix_pol=torch.from_numpy(p.pix_pol).to(dev),
                                                   n_pix_pol=p.n_pix_pol))):
            plan = mm.Plan(pix, psi, p.n_pix, p.interval_offsets, p.interval_filter, lib_lags(p), **kw)
            ops = {}
            for prec in ("fp32", "df64", "fp64"):
                ms, _ = plan.time_operator(prec, reps=20 if prec == "fp32" else 5)
                ops[prec + "_ms"] = float(ms[3])
            skw = dict(precision="mixed", rel_tol=1e-6, max_iter=500, max_outer=10)
            plan.solve(d, **skw)
            ms_s, (m, info) = _timed(lambda: plan.solve(d, **skw), steps)
            res[name] = {"operator": ops, "rows": plan.n_obs, "n_obs_pol": plan.stats["n_obs_pol"],
                         "mixed_solve_to_1e-6": {"ms": ms_s, "iters": info["iters"],
                                                 "value": p.n_samples * info["iters"] / (ms_s / 1e3)}}
            plan.close()
        line.update({"n_samples": p.n_samples, **res,
                     "workload_desc": "IQU, 4 det x 2^22 samples, I on 512x512, Q/U on 256x256 (multi-resolution) "
                                      "against all three on 512x512, intervals 2^16-2^20, n_c=2^14"})
    elif args.workload == "config2-checkpoint":
        # float64 solves of the IQU workload with and without checkpoints every 20 iterations
        # (the paper's default), the state written to host memory by the callback
        p = make_config(2)
        plan = mm.Plan(torch.from_numpy(p.pix).to(dev), torch.from_numpy(p.psi).to(dev), p.n_pix,
                       p.interval_offsets, p.interval_filter, lib_lags(p))
        d = torch.from_numpy(p.d[0]).to(dev)
        kw = dict(precision="fp64", rel_tol=1e-10, max_iter=200)
        plan.solve(d, **kw)
        ms0, (m0, i0) = _timed(lambda: plan.solve(d, **kw), steps)
        saved = []

        def keep(state):
            saved.append(state["iters"])
            return False

        plan.solve(d, checkpoint_every=20, on_checkpoint=keep, **kw)
        saved.clear()
        ms1, (m1, i1) = _timed(lambda: plan.solve(d, checkpoint_every=20, on_checkpoint=keep, **kw), steps)
        n_ck = len(saved) // max(steps, 1)
        diff = float((m1 - m0).norm() / m0.norm())
        line.update({"n_samples": p.n_samples, "iters": i0["iters"], "ms_without": ms0, "ms_with": ms1,
                     "checkpoints_per_solve": n_ck,
                     "ms_per_checkpoint": (ms1 - ms0) / max(n_ck, 1), "map_rel_diff": diff,
                     "checkpoint_bytes": 5 * plan.n_obs * 3 * 8,
                     "workload_desc": "IQU workload, float64 solve to rel. residual 1e-10, checkpoints every 20 "
                                      "iterations (five maps and six scalars to host memory)"})
        plan.close()
    elif args.workload == "config2-boresight":
        # the same scan planned twice: pointing expanded on the fly from the
        # boresight nodes, and the expansion stored per sample
        from synth.boresight import make_boresight_config2
        p = make_boresight_config2()
        otf = mm.Plan.from_boresight(torch.from_numpy(p.boresight).to(dev), p.bore_step, p.det, p.samples_per_det,
                                     p.width, p.height, True, p.interval_offsets, p.interval_filter, lib_lags(p))
        if args.operator_only:      # a short run of the on-the-fly float32 operator alone (for ncu)
            ms, n = otf.time_operator("fp32", reps=args.operator_only)
            print(json.dumps({"operator_only": "config2-boresight on the fly", "fp32_ms": [float(x) for x in ms],
                              "launches": [int(x) for x in n]}), flush=True)
            otf.close()
            return
        pix, c2, s2 = otf.expand_pointing()
        psi = (0.5 * torch.atan2(s2.double(), c2.double())).float()
        stored = mm.Plan(pix, psi, p.n_pix, p.interval_offsets, p.interval_filter, lib_lags(p))
        del pix, c2, s2, psi
        d = torch.from_numpy(p.d[0]).to(dev)
        res = {}
        for name, plan in (("stored", stored), ("on_the_fly", otf)):
            ops = {}
            for prec in ("fp32", "df64", "fp64"):
                ms, _ = plan.time_operator(prec, reps=20 if prec == "fp32" else 5)
                ops[prec + "_ms"] = float(ms[3])
                if prec == "fp32":
                    ops["fp32_per_kernel_ms"] = [float(x) for x in ms[:3]]
            kw = dict(precision="mixed", rel_tol=1e-6, max_iter=500, max_outer=10)
            plan.solve(d, **kw)
            ms_s, (m, info) = _timed(lambda: plan.solve(d, **kw), steps)
            res[name] = {"operator": ops, "device_bytes": plan.stats["device_bytes"],
                         "mixed_solve_to_1e-6": {"ms": ms_s, "iters": info["iters"],
                                                 "value": p.n_samples * info["iters"] / (ms_s / 1e3)},
                         "n_obs": plan.n_obs}
        line.update({"n_samples": p.n_samples, "bore_step": p.bore_step, "n_bore": int(p.boresight.shape[0]),
                     "fft_len": otf.stats["fft_len"], **res,
                     "operator_fp32_speedup_on_the_fly": res["stored"]["operator"]["fp32_ms"]
                     / res["on_the_fly"]["operator"]["fp32_ms"],
                     "workload_desc": "IQU, 4 det x 2^22 samples, 512x512 grid, overshooting raster with off-grid "
                                      "turnarounds, boresight nodes every 16 samples, focal plane turning once per "
                                      "4 sweeps, intervals 2^16-2^20, n_c=2^14"})
        stored.close()
        otf.close()
    else:
        p = make_config(5)
        plan = mm.Plan(torch.from_numpy(p.pix).to(dev), torch.from_numpy(p.psi).to(dev), p.n_pix,
                       p.interval_offsets, p.interval_filter, lib_lags(p))
        d = torch.from_numpy(p.d[0]).to(dev)
        o2g, exc = plan.observed()
        keep = torch.from_numpy(~exc.cpu().numpy().astype(bool)).to(dev)
        target = torch.from_numpy(p.target[o2g.cpu().numpy()]).to(dev)
        kw = dict(precision="mixed", rel_tol=1e-8, max_iter=500, max_outer=10)

        def step():
            params = torch.tensor(p.noise_params, dtype=torch.float64, requires_grad=True)
            dd = d.clone().requires_grad_(True)
            m = mm.MadmapSolve.apply(dd, params, plan, p.fs, kw)
            loss = ((m - target) ** 2)[keep].sum()
            loss.backward()
            return params.grad

        for _ in range(warm):
            step()
        ms, _ = _timed(step, steps)
        fwd_ms, (m, info) = _timed(lambda: plan.solve(d, **kw), steps)
        g = 2.0 * (m - target) * keep[:, None]
        bwd_ms, (_, _, binfo) = _timed(lambda: plan.solve_backward(d, m, g.contiguous(), rel_tol=1e-8), steps)
        line.update({"n_samples": p.n_samples, "ms_forward_backward": ms, "ms_forward": fwd_ms, "ms_backward": bwd_ms,
                     "forward_iters": info["iters"], "adjoint_iters": binfo["iters"],
                     "workload_desc": "IQU, 16 det x 2^22, 256x256, n_c=2^12; loss |m - t|^2; grads wrt d and "
                                      "(sigma, f_knee, alpha) per detector"})
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- headline
def headline_problem(workload, rank, dev, n_det=32):
    """(problem, pix, psi, d) with pix, psi, d on the device."""
    import torch
    if workload == "config3":
        from synth.allsky import make_allsky_problem
        p = make_allsky_problem(scale=0, n_det=n_det, device=dev, seed=3000 + rank)
        return p, p.pix, p.psi, p.d[0]
    from synth import make_config
    p = make_config(2, seed=2000 + rank)
    return (p, torch.from_numpy(p.pix).to(dev), torch.from_numpy(p.psi).to(dev),
            torch.from_numpy(p.d[0]).to(dev))


def oracle_reference_map(p, plan):
    """The FP64 oracle's PCG map (relative residual 1e-12) over the plan's observed pixels."""
    import numpy as np

    from oracle.noise import filter_lags
    from oracle.solver import System
    lags = np.stack([filter_lags(p.n_lags, p.fs, *p.noise_params[k]) for k in range(p.n_filters)])
    S = System(p.pix, p.psi, p.n_pix, p.n_stokes, p.interval_offsets, p.interval_filter, lags)
    o2g, exc = plan.observed()
    if not (np.array_equal(o2g.cpu().numpy().astype(np.int64), S.obs2glob)
            and np.array_equal(exc.cpu().numpy().astype(bool), S.excised)):
        raise RuntimeError("the plan's observed pixels differ from the oracle's")
    t0 = time.perf_counter()
    x, info = S.solve(p.d[0], rel_tol=1e-12, max_iter=3000)
    return x, ~S.excised, (f"FP64 oracle PCG solve to relative residual 1e-12 ({info['iters']} iterations, "
                           f"{time.perf_counter() - t0:.0f} s on one host core)")


def first_tol(solve_err):
    """Loosest tolerance of TOLS whose map error is within MAP_TARGET, by bisection
    (the error falls as the tolerance tightens).  solve_err(tol) -> (info, err, per);
    returns (tol, info, err, per), the tightest tolerance if none reaches it."""
    cache = {}

    def ev(i):
        if i not in cache:
            cache[i] = solve_err(TOLS[i])
        return cache[i]

    lo, hi = 0, len(TOLS) - 1
    if ev(hi)[1] > MAP_TARGET:
        return (TOLS[hi],) + ev(hi)
    while lo < hi:
        mid = (lo + hi) // 2
        if ev(mid)[1] <= MAP_TARGET:
            hi = mid
        else:
            lo = mid + 1
    return (TOLS[hi],) + ev(hi)


def run_headline(args, world, rank, local):
    import numpy as np
    import torch

    import paper_0906_1775_gb300 as mm

    workload = args.workload
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mm.load()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    # one independent replica per rank (weak scaling, no data-path collective)
    t0 = time.time()
    p, pix, psi, d = headline_problem(workload, rank, dev, args.det)
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    t0 = time.time()
    plan = mm.Plan(pix, psi, p.n_pix, p.interval_offsets, p.interval_filter, lib_lags(p), tiles_per_chunk=args.tpc,
                   fft_len=args.fft_len, autotune=not args.no_autotune, scatter_runs=args.scatter_runs,
                   fft_split=args.fft_split)
    torch.cuda.synchronize()
    plan_s = time.time() - t0
    n_obs = plan.n_obs
    if args.operator_only:
        ms, n = plan.time_operator("fp32", reps=args.operator_only)
        ms64, _ = plan.time_operator("fp64", reps=max(1, args.operator_only // 4))
        msdf, _ = plan.time_operator("df64", reps=max(1, args.operator_only // 4))
        print(json.dumps({"workload": workload, "operator_fp32_ms_per_launch": list(ms[:3]),
                          "launches": [int(x) for x in n], "operator_fp32_ms": float(ms[3]),
                          "operator_fp32_sequential_ms": float((ms[:3] * n).sum()),
                          "operator_fp64_ms": float(ms64[3]), "operator_df64_ms": float(msdf[3]),
                          "operator_df64_ms_per_launch": list(msdf[:3]), "stats": plan.stats}), flush=True)
        plan.close()
        return
    sample = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = detector_sample(p, 0, pix, psi, d)
    del pix, psi
    if args.profile_step > 0:
        _, info = plan.solve(d, precision="mixed", rel_tol=args.profile_step, max_iter=3000, max_outer=30,
                             use_graph=args.profile_graph, inner_rel_tol=args.inner_tol)
        torch.cuda.synchronize()
        print(json.dumps({"profile_step": info, "launches": mm.madmap_kernel_launch_count()}), flush=True)
        plan.close()
        return

    # ---------------- reference map
    if workload == "config2":
        ref, keep, ref_desc = oracle_reference_map(p, plan)
    else:
        _, exc = plan.observed()
        keep = ~exc.cpu().numpy().astype(bool)
        ref_t, rinfo = plan.solve(d, precision="fp64", rel_tol=1e-11, max_iter=5000)
        ref = ref_t.cpu().numpy()
        del ref_t
        ref_desc = (f"float64 GPU PCG solve to relative residual 1e-11 ({rinfo['iters']} iterations); the float64 "
                    f"operator and solve are checked against the FP64 oracle in the tests")

    def solve_err(precision, **kw):
        def f(tol):
            m, info = plan.solve(d, precision=precision, rel_tol=tol, max_iter=5000, **kw)
            err, per = stokes_err(m.cpu().numpy(), ref, keep)
            return info, err, per
        return f

    def time_solve(precision, tol, **kw):
        plan.solve(d, precision=precision, rel_tol=tol, max_iter=5000, **kw)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        plan.solve(d, precision=precision, rel_tol=tol, max_iter=5000, **kw)
        t1.record()
        torch.cuda.synchronize()
        return t0.elapsed_time(t1)

    # mixed precision: the inner float32 tolerance is a free parameter of the
    # method; the fastest setting that reaches the map error is timed
    best_mixed = None
    for inner in (1e-4, 3e-5, 1e-5, 3e-6):
        kw_i = dict(max_outer=30, inner_rel_tol=inner)
        cand = first_tol(solve_err("mixed", **kw_i))
        if cand[2] > MAP_TARGET:
            continue
        t = time_solve("mixed", cand[0], **kw_i)
        if best_mixed is None or t < best_mixed[0]:
            best_mixed = (t, kw_i, cand)
    if best_mixed is None:
        raise RuntimeError("no mixed-precision setting reached the map error target")
    mixed_kw, (tol_mixed, info_mixed, err_mixed, per_mixed) = best_mixed[1], best_mixed[2]
    tol_64, info_64, err_64, per_64 = first_tol(solve_err("fp64"))

    def solve_step():
        return plan.solve(d, precision="mixed", rel_tol=tol_mixed, max_iter=5000, **mixed_kw)

    for _ in range(max(args.warmup, 0)):
        solve_step()

    # ---------------- timed region
    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        gpu_index = vis.split(",")[local]
    clocks = Clocks(gpu_index)
    time.sleep(0.3)
    launches0 = mm.madmap_kernel_launch_count()
    iters = 0
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        _, info = solve_step()
        iters += info["iters"]
    e1.record()
    torch.cuda.synchronize()
    barrier(world)
    launches = mm.madmap_kernel_launch_count() - launches0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(world, ms, dev)
    samples_iters = sum_over_ranks(world, float(p.n_samples) * iters, dev)
    value = samples_iters / (ms_max / 1e3)

    # ---------------- float64 time to the same map error
    ms_fp64 = time_solve("fp64", tol_64)

    # ---------------- roofline of the float32 operator (events on the kernels' own stream)
    op_ms, op_launch = plan.time_operator("fp32", reps=20)
    op64_ms, _ = plan.time_operator("fp64", reps=3)
    opdf_ms, _ = plan.time_operator("df64", reps=5)
    t_op = float(op_ms[3])            # one application as the solver launches it
    # algorithmic bytes and flops of one application (pointing read once, map read
    # and written; FFT flops at the paper's FFT length, Section 5.2 Eq. 22)
    b_alg = p.n_samples * 8 + 2 * n_obs * 4 * 3
    n_c = p.n_lags
    n_f = mm.paper_fft_length(n_c, int(np.diff(p.interval_offsets).max()))
    f_per_sample = (5.0 * n_f * np.log2(n_f) + n_f) / (n_f - 2 * n_c)
    f_alg = p.n_samples * f_per_sample
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12     # FP32 FMA lanes x 2 x clock
    achieved_tf = f_alg / (t_op * 1e-3) / 1e12
    achieved_gbs = b_alg / (t_op * 1e-3) / 1e9
    k_dom = int(np.argmax(op_ms[:3] * op_launch))
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved_tf / alu_peak, "traffic": None,
                "kernel": "operator A^T N^-1 A, float32: one application = k_f1 (gather + column FFTs), "
                          "k_f2 (row FFTs x filter), k_f3 (inverse column FFTs + scatter) over all tile chunks",
                "alg_flops_per_launch": float(f_alg), "alg_bytes_per_launch": int(b_alg), "ms_per_launch": t_op,
                "peak_source": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 flops x {sm_mhz:.0f} MHz",
                "hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": achieved_gbs / hbm_peak,
                        "peak_source": f"{hbm_peak_src} hbm_gbs (MEASURED_PEAKS.json)"},
                "t_roof_us": {"bytes": b_alg / (hbm_peak * 1e9) * 1e6, "flops": f_alg / (alu_peak * 1e12) * 1e6},
                "per_kernel_ms": [float(x) for x in op_ms[:3]], "launches_per_application": [int(x) for x in op_launch],
                "dominant_kernel": ["k_f1", "k_f2", "k_f3"][k_dom],
                "fp64_operator_ms": float(op64_ms[3]),
                "df64_operator_ms": float(opdf_ms[3])}
    # DRAM traffic per application from the committed ncu summary, used only while
    # the operator source is the one the counters were taken with
    traffic_file = os.path.join(ROOT, "profiles", f"operator_traffic_{workload}.json")
    if os.path.exists(traffic_file):
        try:
            tr = json.load(open(traffic_file))
            if (tr.get("source_sha256") == operator_source_hash() and tr.get("fft_len") == plan.stats["fft_len"]
                    and tr.get("n2") == plan.stats["n2"] and tr.get("n_tiles") == plan.stats["n_tiles"]):
                roofline["traffic"] = tr["dram_bytes_per_application"]
                roofline["traffic_source"] = tr.get("how")
        except Exception:
            pass

    # ---------------- end to end: host d in, host map out, through the public API
    # Every step uploads its timestream from pinned host memory and reads its
    # map back.  The uploads run on a copy stream into two device buffers, so
    # step k+1's upload overlaps step k's solve (a data loader's pattern); the
    # first upload is not hidden.
    d_host = d.cpu().pin_memory()
    m_host = torch.empty((n_obs, 3), dtype=torch.float64).pin_memory()
    dbuf = [torch.empty_like(d), torch.empty_like(d)]
    copy_stream = torch.cuda.Stream(device=dev)
    up = [torch.cuda.Event(), torch.cuda.Event()]
    barrier(world)
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record()
    copy_stream.wait_event(g0)

    def upload(k):
        with torch.cuda.stream(copy_stream):
            dbuf[k % 2].copy_(d_host, non_blocking=True)
            up[k % 2].record(copy_stream)

    e2e_iters = 0
    upload(0)
    for k in range(args.steps):
        if k + 1 < args.steps:
            upload(k + 1)   # its buffer's last reader, step k - 1's solve, has returned
        torch.cuda.current_stream().wait_event(up[k % 2])
        m, info = plan.solve(dbuf[k % 2], precision="mixed", rel_tol=tol_mixed, max_iter=5000, **mixed_kw)
        m_host.copy_(m, non_blocking=True)
        e2e_iters += info["iters"]
    g1.record()
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(world, g0.elapsed_time(g1), dev)
    e2e_value = sum_over_ranks(world, float(p.n_samples) * e2e_iters, dev) / (ms_e2e / 1e3)
    del dbuf, d_host

    cpu = None
    if sample is not None:
        n_proc = args.cpu_procs or min(16, host_cores())
        cpu = cpu_baseline(sample, args.cpu_iters, n_proc, "detector 0's share of this workload "
                           f"({sample['pix'].shape[0]} samples, {len(sample['offsets']) - 1} intervals)")

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": HEADLINE[workload], "n_samples": p.n_samples, "unknowns": int(n_obs * 3),
                           "n_obs": n_obs, "n_excised": plan.stats["n_excised"],
                           "fft_len": plan.stats["fft_len"], "n2": plan.stats["n2"], "n_tiles": plan.stats["n_tiles"],
                           "l2_flush": "inputs larger than L2 (pointing + d = "
                                       f"{p.n_samples * 12 / 1e6:.0f} MB > 129 MB L2)",
                           "replicas": "one independent problem per rank", "generate_s": gen_s,
                           "plan_create_s": plan_s, "device_bytes": plan.stats["device_bytes"],
                           "tiles_per_chunk": plan.stats["tiles_per_chunk"],
                           "scatter_runs": plan.stats["scatter_runs"],
                           "repeat_frac": round(plan.stats["repeat_frac"], 4),
                           "autotune": [{"fft_len": m, "n2": n2, "tiles_per_chunk": t, "fp32_operator_ms": ms, "runs": r}
                                        for m, t, ms, r, n2 in plan.stats["tuned"]]},
                "time_to_1e-6_map_error": {
                    "mixed_ms": ms_max / args.steps, "mixed_iters": iters // max(args.steps, 1),
                    "mixed_rel_tol": tol_mixed, "mixed_map_err": err_mixed, "mixed_map_err_IQU": per_mixed,
                    "mixed_outer": info_mixed["outer_iters"], "mixed_inner_rel_tol": mixed_kw["inner_rel_tol"],
                    "fp64_ms": ms_fp64, "fp64_iters": info_64["iters"], "fp64_rel_tol": tol_64,
                    "fp64_map_err": err_64, "fp64_map_err_IQU": per_64,
                    "speedup_mixed_vs_fp64": ms_fp64 / (ms_max / args.steps),
                    "reference": ref_desc},
                "roofline": roofline,
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(p.n_samples * 4),
                        "d2h_bytes_per_step": int(n_obs * 3 * 8),
                        "copies": "pinned host timestream uploaded every step on a copy stream (step k+1's "
                                  "upload overlaps step k's solve), map read back every step"},
                "gpu_launches": int(launches),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    plan.close()


# ----------------------------------------------------------------------------- main
def main():
    args = parse()
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload in HEADLINE:
        run_headline(args, world, rank, local)
    elif rank == 0:
        run_secondary(args)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
