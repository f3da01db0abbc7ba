#!/usr/bin/env python3
"""Benchmark: cell-direction-step updates/s of the time-dependent RT forward model.

Workload: the phantom-scale homogeneous slab (96 x 96 x 64 voxels at 1 mm, 192 HEALPix
directions, mu_a 0.008/mm, mu_s 8/mm, g 0.9, n 1.4, 15-degree delta pulse at the centre
of the -z face, 8 detectors, 10 ps bins).  A bench "step" is one time step of the whole
path (sweep, source iteration, detector / energy tallies).  The solve is spun up from
the pulse for --spinup steps (untimed) so that the timed window lies inside the
developed part of the 1500-step solve; then --warmup steps, then --steps timed steps
with CUDA events on the library's stream.  The ring history (4.5 GB) is far larger
than L2, so no L2 flush is needed between steps.

Keys beyond the base contract: "roofline" (the dominant kernel against the measured
peak), "kernels" (all kernels), "cpu_baseline" (the FP64 oracle timed on the host on a
bounded voxel sample), "e2e" (the whole job through the public API from host buffers),
"clocks" (nvidia-smi samples during the timed window), "iterations" (source-iteration
statistics of the window), and one object per other measured workload, each with its
own time per step, roofline and clocks: "fp32" (the plain-FP32 path on the same slab and
window), "config1" (16^3 voxels, 48 directions, 100 graph-replayed steps, plain FP32 and
BF16-scatter), "config3" (the 128 x 128 x 96 heterogeneous phantom with Fresnel
interfaces, BF16 scatter and FP32 sweep, on the general per-voxel kernel forms).

--impl reference times the oracle alone (see CpuLeg) on the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}
METRIC = "cell*dir*step updates/s"
FP32_LANES_PER_SM = 128


def sm_count():
    """Streaming multiprocessors of the device the bench runs on (queried, not assumed)."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def fp32_peak_tflops(pk):
    """FP32 FFMA peak: SMs x 128 FP32 lanes x 2 FLOP x the measured maximum SM clock."""
    return sm_count() * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            p = json.load(f)
        p["_source"] = "measured"
        return p
    except (OSError, ValueError):
        p = dict(FALLBACK_PEAKS)
        p["_source"] = "fallback"
        return p


def measured_traffic(kernel, updates):
    """DRAM bytes of one launch of ``kernel`` from the committed ncu table, scaled to
    ``updates`` (traffic grows in proportion to the updates a launch processes), or None
    when the kernel's source has changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        parts = ln.split()
        if len(parts) >= 4 and not ln.startswith("#") and parts[0] == kernel:
            src = os.path.join(ROOT, "paper_2105_01028_gb300", "csrc", parts[1])
            try:
                sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:len(parts[2])]
            except OSError:
                return None
            return float(parts[3]) * updates if sha == parts[2] else None
    return None


def max_over_ranks(ms):
    """The slowest rank's time (ms) when the bench runs as several ranks (one replica per
    GPU under torch.distributed), else ``ms`` itself."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws, updates_per_rank, ms):
    """Whole-job throughput: the updates of all ``ws`` replicas over the slowest rank's time."""
    return ws * updates_per_rank / (ms * 1e-3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ CPU (oracle) leg

class CpuLeg:
    """The FP64 oracle's work for one time step at a random voxel sample (all
    directions): the upwind gather, Eq. 10 and the per-voxel source iteration, from a
    smooth synthetic developed history (the CPU cannot reach the developed part of the
    solve itself: one full-grid oracle step takes about 30 s).  The oracle's model and the
    history are built once; each sample is timed on its own."""

    def __init__(self, prob, seed=7):
        from oracle.solver import Model
        self.model = Model(dict(prob, tol=prob.get("tol", 1e-6)))
        self.Ih, self.Sh = W.developed_history(prob, seed=seed)
        self.s_glob = float(np.abs(self.Sh[-1]).max())

    def sample(self, n_voxels, seed):
        """(updates/s, info) of one step at ``n_voxels`` random voxels."""
        from oracle.solver import one_step_at
        Ih, Sh = self.Ih, self.Sh
        levels = Ih.shape[0]

        def hist(which, lev, d, u):
            arr = Ih if which == "I" else Sh
            out = np.zeros(np.shape(lev))
            ok = (lev < 0) & (lev >= -levels)
            out[ok] = arr[levels + lev[ok], d[ok], u[ok]]
            return out

        rng = np.random.default_rng(seed)
        vox = np.sort(rng.choice(self.model.nv, n_voxels, replace=False))
        t0 = time.perf_counter()
        _, _, iters = one_step_at(self.model, 0, hist, vox, self.s_glob)
        dt = time.perf_counter() - t0
        return n_voxels * self.model.na / dt, dict(seconds=dt, voxels=int(n_voxels),
                                                   iters_mean=float(np.mean(iters)))


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    nx, ny, nz = args.grid
    prob = W.config_slab(steps=args.spinup + args.warmup + args.steps, nx=nx, ny=ny, nz=nz)
    vals = []
    info = None
    leg = CpuLeg(prob)
    for k in range(args.warmup + args.steps):
        v, info = leg.sample(args.ref_voxels, seed=100 + k)
        if k >= args.warmup:
            vals.append(v)
    value = float(np.mean(vals))
    sample = ("per bench step: one time step of the FP64 oracle at %d random voxels x 192 "
              "directions of the 96x96x64 slab (sweep gather, Eq. 10, source iteration to "
              "tol 1e-6) from a synthetic developed history" % args.ref_voxels)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "updates/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * info["seconds"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, precision="fp64 (oracle)"),
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": cpu_cores(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ GPU leg

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is None:
            self.out = ""
            return
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                try:
                    rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
                except ValueError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, x in enumerate(r) if x.lower() == "active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def workload_config(args, precision=None):
    """The headline workload's description; ``precision`` names the arithmetic of the arm
    that reports it (the reference arm: the FP64 oracle)."""
    nx, ny, nz = args.grid
    if args.two_level:
        dirs = "3072 HEALPix transport dirs (Nside 16), source function on 192 (Nside 4, mean of 16 children)"
        hist = "36 GB"
    else:
        dirs = "192 HEALPix dirs (Nside 4)"
        hist = "4.5 GB"
    return {"workload": "phantom-scale slab %dx%dx%d voxels @1mm, %s, " % (nx, ny, nz, dirs) +
                        "mu_a 0.008/mm, mu_s 8/mm, g 0.9, n 1.4, 15-deg delta pulse, 8 detectors, "
                        "10 ps bins",
            "window": "time steps %d..%d of the 1500-step solve" % (
                args.spinup + args.warmup, args.spinup + args.warmup + args.steps - 1),
            "tol": 1e-6, "l2": "inputs larger than L2 (%s time-level history per solve)" % hist,
            "parallelism": "replicas" if dist_env()[0] > 1 else "single GPU",
            "precision": precision or (("fp32" if args.exact_simt else "3xtf32") if args.exact else args.precision),
            "source_function": (("exact per-voxel solve S = M Q, " +
                                 ("FP32 SIMT products" if args.exact_simt else
                                  "three TF32 tensor-core products with FP32 accumulation"))
                                if args.exact else "source iteration (Eq. 12)")}


def serve_measure(args, n_burst, n_req, rates, seed=4):
    """Served stream (the served workload, a bounded number of requests): cubic grids of
    32..96 voxels, 48 or 192 directions, 500..1500 steps, log-normal random-field optics
    (workloads.served_stream / config_served).  First the capacity is measured: a burst of
    ``n_burst`` requests submitted at once, solves/s over its makespan.  Then for each
    rate factor in ``rates`` a stream of ``n_req`` requests arrives as a Poisson process at
    that fraction of the capacity, each request submitted at its arrival time; reported
    per rate: solves/s over the makespan, p50/p99 latency (submission to detector curves on
    the host), aggregate updates/s and the largest number of concurrent solves."""
    import torch
    import paper_2105_01028_gb300 as T

    def draw(n, sd, rate):
        out = []
        for k, r in enumerate(W.served_stream(n, seed=sd, rate_per_s=rate)):
            p = W.config_served(r["n"], r["nside"], r["steps"], seed=r["seed"], precision=args.precision)
            p["steps"] = r["steps"]
            out.append((r["arrival_s"], p))
        return out

    def updates(reqs):
        return sum(p["nx"] * p["ny"] * p["nz"] * 12 * p["nside"] ** 2 * p["steps"] for _, p in reqs)

    free, total = torch.cuda.mem_get_info()
    srv = T.Server(hbm_budget_bytes=int(0.8 * free), max_slots=args.slots, steps_per_slice=32)
    wid = srv.submit(W.config_served(16, 2, 10, seed=1, precision=args.precision))
    srv.wait(wid)

    def play(reqs, timed_arrivals):
        ids = []
        t0 = time.perf_counter()
        for at, p in reqs:
            if timed_arrivals:
                dt = at - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
            ids.append(srv.submit(p))
        lat = []
        for rid in ids:
            st, rc, det, ms = srv.wait(rid, timeout_s=7200)
            if st != T.REQ_DONE:
                raise RuntimeError("request %d ended in state %d (status %d)" % (rid, st, rc))
            lat.append(ms)
        return time.perf_counter() - t0, np.array(lat)

    with ClockSampler(0) as clk:
        burst = draw(n_burst, 40, 1.0)
        span, blat = play(burst, False)
        capacity = len(burst) / span
        c0 = srv.stats()["max_concurrent"]
        results = []
        for f in rates:
            reqs = draw(n_req, seed, f * capacity)
            span, lat = play(reqs, True)
            st = srv.stats()
            results.append({"rate_factor": f, "arrival_rate_per_s": f * capacity, "requests": len(reqs),
                            "solves_per_s": len(reqs) / span, "makespan_s": span,
                            "latency_ms": {"p50": float(np.percentile(lat, 50)),
                                           "p99": float(np.percentile(lat, 99)), "max": float(np.max(lat))},
                            "updates_per_s": updates(reqs) / span, "max_concurrent_so_far": st["max_concurrent"]})
    stats = srv.stats()
    srv.close()
    head = results[-1]
    return {"metric": "served solves/s", "value": head["solves_per_s"], "unit": "solves/s",
            "higher_is_better": True, "precision": args.precision, "data": "synthetic",
            "config": {"workload": "served stream: cubic 32..96 voxels @1mm, 48/192 dirs (p = 1/2), 500..1500 "
                                   "steps, log-normal GRF optics (sigma 0.3, correlation 5 mm, median mu_a "
                                   "0.01/mm, mu_s 10/mm), g 0.9, n 1.4; Poisson arrivals at the stated "
                                   "fractions of the measured capacity; %d requests per rate (bounded "
                                   "sample of the 2000-request stream)" % n_req,
                       "slots": args.slots, "steps_per_slice": 32},
            "capacity": {"solves_per_s": capacity, "burst_requests": len(burst), "makespan_s": len(burst) / capacity,
                         "updates_per_s": updates(burst) * capacity / len(burst), "max_concurrent": c0,
                         "burst_latency_ms": {"p50": float(np.percentile(blat, 50)),
                                              "p99": float(np.percentile(blat, 99))}},
            "rates": results, "latency_ms": head["latency_ms"],
            "max_concurrent": stats["max_concurrent"], "completed": stats["completed"], "clocks": clk.summary()}


def run_serve(args):
    """The served stream alone (--serve N): capacity from a burst of --serve-burst requests,
    then N requests per rate factor in --rates."""
    import torch
    torch.cuda.set_device(0)
    line = serve_measure(args, args.serve_burst, args.serve, args.rates)
    line["n_gpus"] = 1
    print(json.dumps(line))


def run_adjoint(args):
    """Gradient workload (--adjoint): 64^3 voxels, 192 directions, 800 steps, 8 detectors,
    log-normal random-field optics; least-squares misfit between its detector curves and
    those of a map with a 20 % mu_a blob; gradient with respect to mu_a and mu_s per voxel
    by the checkpointed forward (every 50 steps) and the reverse sweep, FP32 with FP64
    sums.  value = cell*dir*step updates per second of the whole gradient (forward +
    reverse, device time); e2e = the same through the public API from host buffers; the
    gradient is checked against a central difference, along a random smooth direction
    through every voxel, of sum G E(mu) with the residual G frozen (two more forward
    solves, untimed)."""
    import torch
    import paper_2105_01028_gb300 as T
    torch.cuda.set_device(0)
    n, steps, every = args.adjoint_grid, args.adjoint_steps, 50
    p, q = W.config_adjoint(n=n, steps=steps)
    nv, na = n ** 3, 12 * p["nside"] ** 2
    stream = torch.cuda.Stream()
    fq = T.Forward(q, stream=stream.cuda_stream)
    fq.run(steps)
    fq.sync()
    obs = fq.detectors()
    fq.close()
    # first-use costs (library load, module load, allocator) on a small case
    pw, _ = W.config_adjoint(n=16, steps=20)
    fw = T.Forward(pw, stream=stream.cuda_stream)
    fw.run_checkpointed(20, 10)
    fw.adjoint(fw.detectors())
    fw.close()
    torch.cuda.synchronize()

    t_job0 = time.perf_counter()
    fw = T.Forward(p, stream=stream.cuda_stream)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with ClockSampler(0) as clk:
        e[0].record(stream)
        fw.run_checkpointed(steps, every)
        e[1].record(stream)
        det = fw.detectors()
        G = det - obs
        e[2].record(stream)
        ga, gs, st = fw.adjoint_profile(G)
        e[3].record(stream)
        stream.synchronize()
    t_job = time.perf_counter() - t_job0
    status = int(fw.last_status)
    ms_fwd = e[0].elapsed_time(e[1])
    ms_adj = e[2].elapsed_time(e[3])
    fit, fit_mean = fw.iterations()
    fw.close()
    L = 0.5 * float(np.sum(G * G))

    # directional central difference through every voxel (untimed), of sum G E(mu) with
    # the residual G frozen: the same gradient J^T G without the misfit's curvature
    rng = np.random.default_rng(8)
    da = W.gaussian_random_field(p["mua"].shape, 3.0, 1.0, rng).astype(np.float32)
    ds = W.gaussian_random_field(p["mus"].shape, 3.0, 1.0, rng).astype(np.float32)
    t = 3e-3
    Ls = []
    for sgn in (1.0, -1.0):
        pp = dict(p, mua=(p["mua"] * (1 + sgn * t * da)).astype(np.float32),
                  mus=(p["mus"] * (1 + sgn * t * ds)).astype(np.float32))
        f = T.Forward(pp, stream=stream.cuda_stream)
        f.run(steps)
        f.sync()
        Ls.append(float(np.sum(G * f.detectors())))
        f.close()
    fd = (Ls[0] - Ls[1]) / (2 * t)
    ad = float(np.sum(ga * (p["mua"] * da).ravel()) + np.sum(gs * (p["mus"] * ds).ravel()))

    pk = peaks()
    fp32_peak = fp32_peak_tflops(pk)
    hbm = pk["hbm_gbs"]
    upd = nv * na * steps
    it_adj = float(st[6])
    solve_flops = 2.0 * na * na * nv * it_adj * steps
    solve_ach = solve_flops / (st[3] * 1e-3) / 1e12
    push_bytes = nv * na * 52.0 * steps  # Qpre 4, I/S at two levels 16, Ibar/Sbar RMW 32
    push_ach = push_bytes / (st[4] * 1e-3) / 1e9
    copy_bytes = nv * na * 16.0 * steps  # I and S of every level read and written once
    copy_ach = copy_bytes / (st[2] * 1e-3) / 1e9
    fwd_flops = 2.0 * na * na * nv * float(np.mean(fit_mean)) * steps
    phases = [
        {"name": "forward, checkpointed (sweep + scatter_fp32 + tallies)", "ms": ms_fwd},
        {"name": "checkpoint restores", "ms": st[0]},
        {"name": "recomputed forward steps", "ms": st[1]},
        {"name": "segment-store copies", "ms": st[2], "bound": "hbm", "achieved": copy_ach, "peak": hbm,
         "unit": "GB/s", "frac": copy_ach / hbm},
        {"name": "adj_scatter_fp32 (transposed solve) + injection", "ms": st[3], "bound": "alu",
         "achieved": solve_ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": solve_ach / fp32_peak,
         "iterations_mean": it_adj},
        {"name": "adj_push (+ transposed interface split)", "ms": st[4], "bound": "hbm",
         "achieved": push_ach, "peak": hbm, "unit": "GB/s", "frac": push_ach / hbm,
         "algorithmic_bytes_per_update": 52},
        {"name": "gradient finish", "ms": st[5]},
    ]
    tot = ms_fwd + ms_adj
    for ph in phases:
        ph["share"] = ph["ms"] / tot
    line = {"metric": "adjoint gradient cell*dir*step updates/s", "value": upd / (tot * 1e-3),
            "unit": "updates/s", "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": tot,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "gradient: %d^3 voxels @1mm, 192 HEALPix dirs, %d time steps, 8 "
                                   "detectors, log-normal GRF optics (mu_a 0.01, mu_s 10 /mm), misfit "
                                   "against a 20%% mu_a blob, checkpoints every %d steps" % (n, steps, every),
                       "step": "one bench step = one whole gradient (forward with checkpoints + reverse sweep)",
                       "l2": "inputs larger than L2 (%.1f GB of checkpoints and segment store)"
                             % (T.adjoint_footprint_bytes(p, steps, every) / 1e9)},
            "gpu_launches": int(8 * steps + 3 * steps + (steps + every - 1) // every + 2),
            "status": status,
            "roofline": {"kernel": "adj_scatter_fp32", "bound": "alu", "achieved": solve_ach,
                         "peak": fp32_peak, "unit": "TFLOP/s", "frac": solve_ach / fp32_peak,
                         "traffic": measured_traffic("adj_scatter_fp32_kernel", nv * na),
                         "peak_source": "FP32 FFMA: %d SMs x 128 lanes x 2 x max SM clock" % sm_count()},
            "phases": phases,
            "forward_scatter_tflops": fwd_flops / (ms_fwd * 1e-3) / 1e12,
            "misfit": L, "grad_max": {"mua": float(np.abs(ga).max()), "mus": float(np.abs(gs).max())},
            "fd_check": {"direction": "smooth random field (std 3 mm) on both maps, 0.3 % amplitude; "
                                      "differences of sum G E(mu) with the residual G frozen",
                         "central_difference": fd, "adjoint": ad, "rel_err": abs(fd - ad) / abs(ad)},
            "clocks": clk.summary(),
            "e2e": {"value": upd / t_job, "unit": "updates/s",
                    "what": "whole gradient from host buffers: context + optics upload, checkpointed "
                            "forward, curves read back, dL/dE up, reverse sweep, gradients read back",
                    "h2d_bytes_per_step": 3 * nv * 4 + G.size * 8,
                    "d2h_bytes_per_step": det.size * 8 + 2 * nv * 8}}
    print(json.dumps(line))


def iteration_bound(flops, nbytes, ms, c_bound, c_ach, c_peak, hbm):
    """Roofline of a source-iteration kernel: its algorithmic FLOP per algorithmic byte
    against the ridge point (compute peak / HBM peak) decides whether the compute or the
    HBM roofline bounds it; both fractions are reported."""
    ai = flops / nbytes
    ridge = c_peak * 1e12 / (hbm * 1e9)
    m_ach = nbytes / (ms * 1e-3) / 1e9
    extra = {"arithmetic_intensity": ai, "ridge_flop_per_byte": ridge, "algorithmic_bytes": nbytes,
             "compute_frac": c_ach / c_peak, "hbm_frac": m_ach / hbm}
    if ai >= ridge:
        return c_bound, c_ach, c_peak, "TFLOP/s", extra
    return "hbm", m_ach, hbm, "GB/s", extra


def kernel_roofline(nv, na, na_s, kms, kp, k_mean, precision, pk, exact=None):
    """Per-kernel times (ms per step) and the roofline object of the dominant kernel from
    ``kp`` profiled steps (``kms``: summed ms of sweep, source function, tallies).
    ``exact``: None (the source iteration), "tc" or "simt" (the exact solve's form)."""
    hbm = pk["hbm_gbs"]
    sweep_bytes = nv * na * 20 + nv * 8  # I,S at two levels read (16 B), Q written (4 B); optics
    # Q, S(n-1), S(n-2) read (the extrapolated start), I and S written; optics
    scat_bytes = nv * na_s * 20 + nv * 12
    scat_flops = 2.0 * na_s * na_s * nv * (1.0 if exact else k_mean)
    per = [kms[0] / kp, kms[1] / kp, kms[2] / kp]
    tot = sum(per)
    s_name = ("exact_" + ("tc" if exact == "tc" else "fp32")) if exact else "scatter_" + precision
    extra = {}
    if exact == "tc":
        # one product per voxel, HBM-bound: Q in, I and S out (12 B per update) + class,
        # index and optics bytes per voxel; the tensor pipe runs three TF32 products
        s_bound, s_peak, s_unit = "hbm", hbm, "GB/s"
        x_bytes = nv * na_s * 12 + nv * 5
        s_ach = x_bytes / (per[1] * 1e-3) / 1e9
        tf32_peak = pk.get("bf16_tflops", 1900.0) * 1.1 / 2.25  # measured BF16 x nominal TF32/BF16
        tc_tf = 3 * scat_flops / (per[1] * 1e-3) / 1e12
        extra = {"algorithmic_bytes": x_bytes, "tensor_tflops_3xtf32": tc_tf,
                 "tensor_frac_of_tf32": tc_tf / tf32_peak,
                 "tf32_peak": "%.0f TFLOP/s (measured BF16 burst x 1.1/2.25 nominal ratio)" % tf32_peak}
    else:
        if precision == "bf16" and not exact:
            s_bound, s_peak = "tensor", pk.get("bf16_tflops_sustained", 1700.0)
        else:
            s_bound, s_peak = "alu", fp32_peak_tflops(pk)
        s_unit = "TFLOP/s"
        s_ach = scat_flops / (per[1] * 1e-3) / 1e12
        if not exact:
            s_bound, s_ach, s_peak, s_unit, extra = iteration_bound(scat_flops, scat_bytes, per[1], s_bound,
                                                                    s_ach, s_peak, hbm)
    w_ach = sweep_bytes / (per[0] * 1e-3) / 1e9
    kernels = [
        {"name": "sweep", "ms": per[0], "share": per[0] / tot, "bound": "hbm", "achieved": w_ach,
         "peak": hbm, "unit": "GB/s", "frac": w_ach / hbm, "algorithmic_bytes": sweep_bytes},
        dict({"name": s_name, "ms": per[1], "share": per[1] / tot,
              "bound": s_bound, "achieved": s_ach, "peak": s_peak, "unit": s_unit, "frac": s_ach / s_peak,
              "algorithmic_flops": scat_flops, "hbm_gbs": scat_bytes / (per[1] * 1e-3) / 1e9}, **extra),
        {"name": "tally+advance", "ms": per[2], "share": per[2] / tot},
    ]
    dom = max(kernels[:2], key=lambda k: k["ms"])
    roof = {"kernel": dom["name"], "bound": dom["bound"], "achieved": dom["achieved"], "peak": dom["peak"],
            "unit": dom["unit"], "frac": dom["frac"], "traffic": None,
            "peak_source": pk["_source"] + (" (FP32 FFMA: %d SMs x 128 lanes x 2 x max SM clock)" % sm_count()
                                            if dom["bound"] == "alu" else "")}
    return kernels, roof


def measure_window(T, torch, prob, stream, spinup, warmup, steps, what, slab_traffic=True):
    """One more workload for the bench line: spin the solve up for ``spinup`` steps, run
    ``warmup`` more, then time ``steps`` graph-replayed steps with CUDA events on the
    library's stream (clocks sampled meanwhile), and time up to 10 further steps kernel
    by kernel.  Returns its sub-object."""
    fwd = T.Forward(prob, stream=stream.cuda_stream)
    fwd.run(spinup + warmup)
    fwd.sync()
    first = fwd.steps_done()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        ev0.record(stream)
        fwd.run(steps)
        ev1.record(stream)
        stream.synchronize()
    ms = ev0.elapsed_time(ev1)
    status = fwd.sync()
    it_max, it_mean = fwd.iterations()
    kp = min(steps, 10)
    kms = fwd.profile(kp)
    _, k_it_mean = fwd.iterations()
    executed = fwd.executed_iterations()[first:first + steps]
    kps = fwd.kernels_per_step()
    xform = fwd.exact_form()
    sform = fwd.sweep_form()
    fwd.close()
    nv = prob["nx"] * prob["ny"] * prob["nz"]
    na = 12 * prob["nside"] ** 2
    prec = prob.get("precision", "fp32")
    kernels, roof = kernel_roofline(nv, na, na, kms, kp, float(np.mean(k_it_mean[-kp:])), prec, peaks(),
                                    exact=xform)
    # measured DRAM bytes of the dominant kernel (committed ncu table, captured on the slab,
    # while its source is unchanged); not for workloads whose kernel instances differ
    names = {"sweep": {"tma": "sweep_tma_kernel", "plain": "sweep_kernel"}.get(sform, "sweep2_kernel"),
             "exact_tc": "exact_tc_kernel", "exact_fp32": "exact_gemm192_kernel",
             "scatter_bf16": "scatter_tc_kernel", "scatter_fp32": "scatter_fp32_kernel"}
    if slab_traffic and roof["kernel"] in names:
        roof["traffic"] = measured_traffic(names[roof["kernel"]], nv * na)
    return {"workload": what, "precision": prec, "value": nv * na * steps / (ms * 1e-3), "unit": "updates/s",
            "ms_per_step": ms / steps, "window": "time steps %d..%d" % (first, first + steps - 1),
            "iterations": {"mean": float(np.mean(it_mean[first:first + steps])),
                           "max": int(np.max(it_max[first:first + steps])),
                           "executed_per_voxel": float(np.mean(executed))},
            "status": int(status), "gpu_launches": kps * steps, "roofline": roof, "kernels": kernels,
            "clocks": clk.summary()}


def measure_whole_run(T, torch, prob, stream, steps, what, repeats=5):
    """A short solve timed whole, from step 0 (context set up and warmed beforehand): the
    best of ``repeats`` runs of ``steps`` graph-replayed steps after a reset."""
    fwd = T.Forward(prob, stream=stream.cuda_stream)
    fwd.run(steps)  # first use: graph capture, module load
    fwd.sync()
    best = None
    with ClockSampler(0) as clk:
        for _ in range(repeats):
            fwd.reset()
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            fwd.run(steps)
            ev1.record(stream)
            stream.synchronize()
            ms = ev0.elapsed_time(ev1)
            best = ms if best is None else min(best, ms)
    status = fwd.sync()
    it_max, it_mean = fwd.iterations()
    fwd.reset()
    kms = fwd.profile(steps)
    _, k_it_mean = fwd.iterations()
    kps = fwd.kernels_per_step()
    fwd.close()
    nv = prob["nx"] * prob["ny"] * prob["nz"]
    na = 12 * prob["nside"] ** 2
    prec = prob.get("precision", "fp32")
    kernels, roof = kernel_roofline(nv, na, na, kms, steps, float(np.mean(k_it_mean)), prec, peaks())
    return {"workload": what, "precision": prec, "value": nv * na * steps / (best * 1e-3), "unit": "updates/s",
            "ms_per_step": best / steps, "steps": steps,
            "timing": "whole %d-step solve from step 0, best of %d (CUDA events; graph replay)" % (steps, repeats),
            "iterations": {"mean": float(np.mean(it_mean)), "max": int(np.max(it_max))},
            "status": int(status), "gpu_launches": kps * steps, "roofline": roof, "kernels": kernels,
            "clocks": clk.summary(),
            "l2": "L2-resident (%.1f MB of time-level history): launch- and latency-bound" % (
                2 * 5 * nv * na * 4 / 1e6)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--spinup", type=int, default=600)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--no-fp32", action="store_true",
                    help="skip the plain-FP32 slab on the same window (timed by default)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 16^3 and heterogeneous-phantom workloads (timed by default)")
    ap.add_argument("--cpu-voxels", type=int, default=16384,
                    help="voxels in the CPU-baseline sample of this arm (about 10 s of oracle work)")
    ap.add_argument("--ref-voxels", type=int, default=2048,
                    help="voxels per bench step of --impl reference")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--grid", type=int, nargs=3, default=[96, 96, 64], metavar=("NX", "NY", "NZ"),
                    help="slab size (smaller grids are for profiling captures only)")
    ap.add_argument("--no-serve", action="store_true", help="skip the served-stream sub-object of the default line")
    ap.add_argument("--serve", type=int, default=0, metavar="N",
                    help="run the served stream with N requests per rate instead of the slab")
    ap.add_argument("--serve-burst", type=int, default=12,
                    help="requests of the capacity measurement (submitted at once)")
    ap.add_argument("--rates", type=float, nargs="+", default=[0.5, 0.8, 1.0],
                    help="arrival rates as fractions of the measured capacity")
    ap.add_argument("--slots", type=int, default=8, help="served stream concurrent slots")
    ap.add_argument("--exact", action="store_true",
                    help="exact per-voxel source function (one optics class on the slab) instead of the iteration")
    ap.add_argument("--exact-simt", action="store_true",
                    help="with --exact: the FP32 SIMT form instead of the tensor cores")
    ap.add_argument("--two-level", action="store_true",
                    help="slab on the paper's fiducial angles: 3072 transport, 192 source-function dirs")
    ap.add_argument("--adjoint", action="store_true", help="gradient workload (checkpointed adjoint)")
    ap.add_argument("--adjoint-grid", type=int, default=64)
    ap.add_argument("--adjoint-steps", type=int, default=800)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
        return
    if args.serve:
        run_serve(args)
        return
    if args.adjoint:
        run_adjoint(args)
        return

    import torch
    import paper_2105_01028_gb300 as T
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    total = args.spinup + args.warmup + args.steps + 16
    nx, ny, nz = args.grid
    if args.two_level:
        prob = W.config_slab(steps=total, precision=args.precision, nx=nx, ny=ny, nz=nz, nside=16)
        prob["nside_scatter"] = 4
    else:
        prob = W.config_slab(steps=total, precision=args.precision, nx=nx, ny=ny, nz=nz)
    if args.exact:
        prob["exact"] = "simt" if args.exact_simt else True
    stream = torch.cuda.Stream()
    nv = prob["nx"] * prob["ny"] * prob["nz"]
    na = 12 * prob["nside"] ** 2          # transport directions (updates are counted on these)
    na_s = 12 * (prob.get("nside_scatter") or prob["nside"]) ** 2  # source-function directions
    nch = na // na_s

    # ---- e2e job through the public API, from host buffers: optics upload, spin-up,
    # warm-up and the timed window, per-step tallies and detector curves read back.  The
    # clock sampler runs for the whole job (the GPU is busy throughout), started before
    # and stopped after the job's own clock so that its process start and stop are not
    # counted in the job.
    clk = ClockSampler(local)
    clk.__enter__()
    t_job0 = time.perf_counter()
    fwd = T.Forward(prob, stream=stream.cuda_stream)
    fwd.run(args.spinup)
    fwd.run(args.warmup)
    fwd.sync()
    first = fwd.steps_done()

    # ---- timed window (device time, CUDA events on the library's stream)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    fwd.run(args.steps)
    ev1.record(stream)
    stream.synchronize()
    ms = ev0.elapsed_time(ev1)
    torch.cuda.synchronize()
    status = fwd.sync()
    det = fwd.detectors()
    N, esc = fwd.energy()
    t_job = time.perf_counter() - t_job0
    clk.__exit__(None, None, None)
    ms = max_over_ranks(ms)
    job_steps = fwd.steps_done()
    it_max, it_mean = fwd.iterations()
    win_max = it_max[first:first + args.steps]
    win_mean = it_mean[first:first + args.steps]

    # ---- per-kernel device times (CUDA events around each kernel, right after the window)
    kp = min(args.steps, 10)
    kms = fwd.profile(kp)
    k_it_max, k_it_mean = fwd.iterations()
    k_mean = float(np.mean(k_it_mean[-kp:]))
    executed = fwd.executed_iterations()[first:first + args.steps]
    k_exec = float(np.mean(fwd.executed_iterations()[-kp:]))  # the profiled steps
    kps = fwd.kernels_per_step()
    xform = fwd.exact_form()
    sweep_kernel = {"plain": "sweep_kernel", "tma": "sweep_tma_kernel", "two-level": "sweep2_kernel"}[fwd.sweep_form()]
    fwd.close()

    updates = nv * na * args.steps
    value = job_value(ws, updates, ms)
    pk = peaks()
    hbm = pk["hbm_gbs"]
    if nch == 1:
        sweep_bytes = nv * na * 20 + nv * 8  # I,S at two levels read (16 B), Q written (4 B); optics
    else:
        # fine I at two levels (8 B) and Q written (4 B) per fine update; coarse S at two
        # levels and the coarse mean Q once per coarse update
        sweep_bytes = nv * na * 12 + nv * na_s * 12 + nv * 8
    fin_bytes = nv * na * 8 + nv * na_s * 4 if nch > 1 else 0  # refine: Q_f in, I_f out, S_c in
    # Q, S(n-1), S(n-2) read (the extrapolated start), I and S written; optics
    scat_bytes = nv * na_s * 20 + nv * 12
    scat_flops = 2.0 * na_s * na_s * nv * k_mean  # angular sum per voxel per iteration
    per = [kms[0] / kp, kms[1] / kp, kms[2] / kp]
    tot = sum(per)
    fp32_peak = fp32_peak_tflops(pk)
    if args.precision == "bf16" and not args.exact:
        s_bound, s_peak, s_unit = "tensor", pk.get("bf16_tflops_sustained", 1700.0), "TFLOP/s"
    else:
        s_bound, s_peak, s_unit = "alu", fp32_peak, "TFLOP/s"
    s_ach = scat_flops / (per[1] * 1e-3) / 1e12
    s_name = "exact_fp32" if args.exact else "scatter_" + args.precision
    tc_extra = {}
    if args.exact and xform == "tc":
        # one product per voxel: HBM-bound (Q in, I and S out: 12 B per update, plus the
        # voxel's class, index and optics bytes); the tensor pipe runs three TF32 products
        s_name, s_bound, s_peak, s_unit = "exact_tc", "hbm", hbm, "GB/s"
        x_bytes = nv * na_s * 12 + nv * 5
        s_ach = x_bytes / (per[1] * 1e-3) / 1e9
        tf32_peak = pk.get("bf16_tflops", 1900.0) * 1.1 / 2.25  # measured BF16 x nominal TF32/BF16
        tc_tf = 3 * scat_flops / (per[1] * 1e-3) / 1e12
        tc_extra = {"algorithmic_bytes": x_bytes, "tensor_tflops_3xtf32": tc_tf,
                    "tensor_frac_of_tf32": tc_tf / tf32_peak,
                    "tf32_peak": "%.0f TFLOP/s (measured BF16 burst x 1.1/2.25 nominal ratio)" % tf32_peak}
    elif not args.exact:
        c_peak = s_peak
        s_bound, s_ach, s_peak, s_unit, tc_extra = iteration_bound(scat_flops, scat_bytes, per[1], s_bound, s_ach,
                                                                   s_peak, hbm)
        if args.precision == "bf16" and k_exec > 0:
            # what the tensor pipe executes: every tile iterates until its slowest voxel
            # stops, and X is carried as two BF16 terms (two MMAs per iteration)
            ex_tf = 2 * 2.0 * na_s * na_s * nv * k_exec / (per[1] * 1e-3) / 1e12
            tc_extra.update({"executed_iterations_per_voxel": k_exec, "tensor_tflops_executed": ex_tf,
                             "tensor_frac_executed": ex_tf / c_peak})
    w_ach = sweep_bytes / (per[0] * 1e-3) / 1e9
    kernels = [
        {"name": "sweep", "ms": per[0], "share": per[0] / tot, "bound": "hbm",
         "achieved": w_ach, "peak": hbm, "unit": "GB/s", "frac": w_ach / hbm,
         "algorithmic_bytes": sweep_bytes,
         "traffic": measured_traffic(sweep_kernel, nv * na)},
        dict({"name": s_name, "ms": per[1], "share": per[1] / tot,
              "bound": s_bound, "achieved": s_ach, "peak": s_peak, "unit": s_unit,
              "frac": s_ach / s_peak, "algorithmic_flops": scat_flops,
              "hbm_gbs": scat_bytes / (per[1] * 1e-3) / 1e9}, **tc_extra),
        {"name": "tally+advance", "ms": per[2], "share": per[2] / tot},
    ]
    if nch > 1:
        f_ach = fin_bytes / (per[2] * 1e-3) / 1e9
        kernels[0]["name"] = "sweep2 (fused coarse mean)"
        kernels[2] = {"name": "refine+tally+advance", "ms": per[2], "share": per[2] / tot, "bound": "hbm",
                      "achieved": f_ach, "peak": hbm, "unit": "GB/s", "frac": f_ach / hbm,
                      "algorithmic_bytes": fin_bytes}
    dom = max(kernels[:2], key=lambda k: k["ms"])
    scat_kernel = (("exact_tc_kernel" if xform == "tc" else "exact_gemm192_kernel") if args.exact else
                   "scatter_tc_kernel" if args.precision == "bf16" else "scatter_fp32_kernel")
    traffic = (measured_traffic(scat_kernel, nv * na_s) if dom is kernels[1]
               else measured_traffic(sweep_kernel, nv * na))
    roof = {"kernel": dom["name"], "bound": dom["bound"], "achieved": dom["achieved"],
            "peak": dom["peak"], "unit": dom["unit"], "frac": dom["frac"], "traffic": traffic,
            "peak_source": pk["_source"] + (" (FP32 FFMA: %d SMs x 128 lanes x 2 x max SM clock)" % sm_count()
                                            if dom["bound"] == "alu" else "")}

    line = {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": (("3xtf32-product/f32-sweep" if xform == "tc" else "f32") if args.exact else
                      "f32" if args.precision == "fp32" else "bf16-scatter/f32-sweep"),
            "data": "synthetic", "config": workload_config(args),
            "gpu_launches": kps * args.steps,
            "iterations": {"mean": float(np.mean(win_mean)), "max": int(np.max(win_max)),
                           "executed_per_voxel": float(np.mean(executed))},
            "status": int(status),
            "roofline": roof, "kernels": kernels, "clocks": clk.summary(),
            "e2e": {"value": ws * nv * na * job_steps / t_job, "unit": "updates/s",
                    "what": "whole job from host buffers: context + optics upload, %d steps, "
                            "tallies and detector curves read back" % job_steps,
                    "h2d_bytes_per_step": 3 * nv * 4 / job_steps,
                    "d2h_bytes_per_step": (det.size * 8 + N.size * 16) / job_steps}}

    plain = not (args.two_level or args.exact)
    if plain and args.precision != "fp32" and not args.no_fp32:
        p32 = W.config_slab(steps=total, precision="fp32", nx=nx, ny=ny, nz=nz)
        sub = measure_window(T, torch, p32, stream, args.spinup, args.warmup, args.steps,
                             "the same slab and time window, plain FP32 (source iteration on CUDA cores)")
        sub["value"] *= ws
        sub["bf16_speedup"] = line["value"] / sub["value"]
        line["fp32"] = sub
    if plain and not args.no_configs and args.grid == [96, 96, 64]:
        c1 = {}
        for prec in ("fp32", "bf16"):
            p1 = W.config_small(steps=100, precision=prec)
            c1[prec] = measure_whole_run(T, torch, p1, stream, 100,
                                         "16^3 voxels @1mm, 48 HEALPix dirs (Nside 2), mu_a 0.01/mm, "
                                         "mu_s 10/mm, g 0.9, n 1.4, 15-deg pulse, 4 detectors, 100 steps, "
                                         "tol 1e-6")
        line["config1"] = c1
        p3 = W.config_hetero(steps=args.spinup + args.warmup + args.steps + 16, precision="bf16")
        line["config3"] = measure_window(
            T, torch, p3, stream, args.spinup, args.warmup, args.steps,
            "heterogeneous phantom 128x128x96 @1mm, 192 dirs, slab optics, air cylinder r 5 mm (n 1) with "
            "Fresnel refraction/reflection at its wall, 3 absorbing spheres r 4/6/8 mm (mu_a x2/x3.5/x5), "
            "-x face pulse, 8 detectors; BF16 scatter, FP32 sweep, general per-voxel kernel forms",
            slab_traffic=False)
        pe = W.config_slab(steps=total, precision="fp32", nx=nx, ny=ny, nz=nz)
        pe["exact"] = True
        line["exact"] = measure_window(
            T, torch, pe, stream, args.spinup, args.warmup, args.steps,
            "the same slab and time window with the exact per-voxel source function S = M Q (one optics "
            "class) on the tensor cores: three TF32 products, FP32 accumulation")
    if plain and not args.no_configs and not args.no_serve and rank == 0:
        line["served"] = serve_measure(args, 8, 12, [0.8])

    if args.two_level or args.exact:
        line["cpu_baseline"] = None
        line["cpu_baseline_note"] = "the timed oracle leg samples the one-level iterated step only"
    if rank == 0 and not args.no_cpu and ws >= 1 and not (args.two_level or args.exact):
        v, info = CpuLeg(prob).sample(args.cpu_voxels, seed=100)
        line["cpu_baseline"] = {"value": v, "unit": "updates/s", "cores": cpu_cores(),
                                "kind": "oracle",
                                "sample": "one time step of the FP64 oracle at %d random voxels x 192 "
                                          "directions from a synthetic developed history (%.1f s, "
                                          "%.0f iterations/voxel mean)" % (
                                              info["voxels"], info["seconds"], info["iters_mean"])}
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
