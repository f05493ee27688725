#!/usr/bin/env python3
"""Benchmark of the nonequilibrium-DMFT lattice step on GB300.

One step = one lattice step of a DMFT iteration (all hot-path rows): the
closed-form B_q - S generation, the Dyson solve of every quadrature point,
the FP64 accumulation of G_loc and of the current j(t), for the N_c = 1500
production configuration (U = E = 1, beta = 10, t in [-5, 30], dt = 0.05,
dtau = 0.1, 53 x 53 Gauss-Hermite points = 2809 solves), with a fixed
synthetic self-energy.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="production N_c=1500 (U=1, E=1, beta=10, t in [-5,30], dt=0.05, dtau=0.1, 53x53 points)",
                t_min=-5.0, t_max=30.0, dt=0.05, beta=10.0, dtau=0.1, U=1.0, E=1.0, n_quad=53)
METRIC = "DMFT iterations/s & TFLOP/s at N_c≈1500; mixed+warm-start vs FP64 at 1e-6 err"
DTYPES = {"fp64": "f64", "mixed_fp32": "f32+f64", "mixed_bf16": "bf16x3+f64"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed_bf16", choices=["fp64", "mixed_fp32", "mixed_bf16"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-points", type=int, default=0, help="oracle sample size (0 = 5 x cores)")
    ap.add_argument("--n-quad", type=int, default=0, help="override the quadrature size (profiling runs only)")
    ap.add_argument("--tts", action="store_true",
                    help="time to a converged solution: mixed + learned warm start vs mixed zero start vs FP64")
    ap.add_argument("--tts-train-runs", type=int, default=64)
    ap.add_argument("--tts-eval", type=int, default=4)
    return ap.parse_args()


# ------------------------------------------------------------------ CPU oracle timing


def _oracle_worker(task):
    from oracle import nedmft_oracle as O
    (t_min, t_max, dt, beta, dtau, U, E, sigma, pts) = task
    c = O.contour_grid(t_min, t_max, dt, beta, dtau)
    m = O.Model(U=U, E=E)
    s = O.weighted_sigma(c, sigma)
    acc = 0.0
    for eps, ebar in pts:
        g0 = O.g0_matrix(c, m, eps, ebar)
        acc += float(np.abs(O.dyson_solve(g0, s)).max())
    return acc


class OracleTimer:
    """The oracle, as it stands, on bounded samples of the workload's points, on
    all host cores: one spawned process pool (one BLAS thread per process) that
    lives across warm-up and timed steps."""

    def __init__(self):
        import multiprocessing as mp

        from oracle import nedmft_oracle as O
        from paper_0711_0999_gb300.synth import workload_sigma

        W = WORKLOAD
        self.cores = os.cpu_count() or 1
        self.c = O.contour_grid(W["t_min"], W["t_max"], W["dt"], W["beta"], W["dtau"])
        self.sigma = workload_sigma(self.c.t, self.c.w, W["U"])
        self.eps, self.ebar, _ = O.quadrature_points(W["n_quad"])
        self.nq = len(self.eps)
        for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        self.pool = mp.get_context("spawn").Pool(processes=self.cores)

    def _tasks(self, npts):
        W = WORKLOAD
        idx = np.linspace(0, self.nq - 1, npts).round().astype(int)
        return [(W["t_min"], W["t_max"], W["dt"], W["beta"], W["dtau"], W["U"], W["E"], self.sigma,
                 [(float(self.eps[i]), float(self.ebar[i]))]) for i in idx]

    def warm(self):
        """One point per process, untimed (process start-up, imports, first solve)."""
        self.pool.map(_oracle_worker, self._tasks(self.cores))

    def time(self, npts: int):
        """Lattice steps/s extrapolated from `npts` evenly spread points, the
        processes used, and a description of the sample."""
        tasks = self._tasks(npts)
        t0 = time.perf_counter()
        self.pool.map(_oracle_worker, tasks)
        dt = time.perf_counter() - t0
        used = min(self.cores, npts)
        sample = (f"{npts} of {self.nq} points of the N_c={self.c.n_c} workload (G0 build + solve(I - G0 S, G0) "
                  f"each), {used} processes x 1 BLAS thread, {dt:.1f} s, scaled by {self.nq}/{npts}")
        return (npts / dt) / self.nq, used, sample

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_sample(n_points: int | None = None):
    """One timed sample (default 5 points per host core, about 12 s of CPU work on
    16 cores) after one warm-up round: (lattice steps/s, cores, sample text)."""
    t = OracleTimer()
    try:
        t.warm()
        return t.time(n_points or 5 * t.cores)
    finally:
        t.close()


def reference_points_per_step(cores: int, steps: int) -> int:
    """Points per timed step of the reference arm: 5 per core for up to 5 steps,
    then fewer (never under one per core), so that K steps together stay at about
    25 points per core (about a minute of CPU work) whatever K is."""
    return max(cores, (25 * cores) // max(steps, 5))


# ------------------------------------------------------------------ clocks


class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples: NEDMFT_CLOCKS_DIR if set (to keep them), else the temporary directory
        out = os.environ.get("NEDMFT_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as fh:
            return parse_clocks(fh)


def parse_clocks(lines):
    """Summary of nvidia-smi samples in ClockSampler.FIELDS order: the median SM
    clock, the maximum SM clock, the sample count and every throttle reason seen
    active in any sample; None without a valid sample."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 7:
            continue
        try:
            sm.append(float(parts[0]))
            smax.append(float(parts[1]))
        except ValueError:
            continue
        for name, val in zip(names, parts[3:7]):
            if val.lower().startswith("active"):
                reasons.add(name)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
            "reasons": sorted(reasons)}


# ------------------------------------------------------------------ peaks


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


# DRAM bytes of one Gauss-Jordan update launch (152 matrices at N_c = 1500), from
# an ncu capture of the same kernel on 16 matrices scaled by 152 / 16; to be
# re-taken whenever the update kernel changes
UPDATE_TRAFFIC_BYTES = 727.6e6 * 152 / 16


def roofline_for(precision: str, tflops: float, gbs: float, peaks, src: str, clocks):
    if precision == "mixed_bf16":
        # a rank-W step of the Gauss-Jordan update (W = 256 complex columns at
        # N_c = 1500) does 8 N^2 W flops per 2 N^2 8 B of FP32 complex traffic,
        # W / 2 = 128 flop/B; in bf16x3 every flop is three bf16 products, so the
        # tensor peak for this arithmetic is the bf16 peak / 3 and the balance
        # point (sustained bf16 / 3 over HBM) is ~88 flop/B: the kernel is
        # bound by the tensor cores
        bf16 = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        peak = bf16 / 3.0
        hpeak = peaks["hbm_gbs"]
        return {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                "traffic": UPDATE_TRAFFIC_BYTES,
                "traffic_note": "ncu dram__bytes_read + write of one update launch on 16 matrices (728 MB), "
                                "scaled by 152/16 to the benchmark launch",
                "peak_source": f"sustained bf16 tensor rate / 3 (bf16x3 = three bf16 products per flop), {src}",
                "hbm": {"achieved": gbs, "peak": hpeak, "unit": "GB/s", "frac": gbs / hpeak,
                        "note": "algorithmic read + write of the FP32 complex matrix per step"}}
    mhz = peaks.get("sm_max_mhz", 2070.0)
    if precision == "mixed_fp32":
        peak = 152 * 128 * 2 * mhz * 1e6 / 1e12  # FP32 FMA lanes x 2 flops x clock
        return {"bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                "traffic": None, "peak_source": "152 SMs x 128 FP32 FMA/clk x 2 x max SM clock"}
    peak = 1.25  # nominal FP64 rate of the part
    return {"bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
            "traffic": None, "peak_source": "nominal FP64 1.25 TFLOP/s", "hbm_gbs": gbs}


# ------------------------------------------------------------------ reference arm


def run_reference(args, rank, world):
    if rank != 0:
        return
    steps_per_s = []
    cores = sample = None
    t = OracleTimer()
    try:
        for _ in range(max(args.warmup, 1)):
            t.warm()
        npts = args.cpu_points or reference_points_per_step(t.cores, args.steps)
        for _ in range(args.steps):
            v, cores, sample = t.time(npts)
            steps_per_s.append(v)
    finally:
        t.close()
    v = statistics.median(steps_per_s)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "iterations/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "n_c": 1500, "points": WORKLOAD["n_quad"] ** 2,
                       "parallelism": "host process pool"},
            "cpu_baseline": {"value": v, "unit": "iterations/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ time to solution


def run_tts(args):
    """Converged DMFT at N_c = 1500 (tol 1e-6, the paper's pointwise criterion):
    mixed path from Sigma = 0, mixed path from the learned warm start, and the FP64
    path (one lattice step + one impurity step measured, times the iterations of
    the converged mixed run).  The network is trained on runs shaped like the
    warm-start configuration: U ~ U[0.25, 2.5], E ~ U[0.25, 4] (seed 20071101),
    N_c = 400 (t in [-5, 10], dt = 0.1, dtau = 0.1), 32 x 32 points."""
    import torch

    from paper_0711_0999_gb300 import api, warmstart

    torch.cuda.set_device(0)
    W = WORKLOAD
    tol = 1e-6
    rng = np.random.default_rng(20071101)
    train = list(zip(rng.uniform(0.25, 2.5, args.tts_train_runs), rng.uniform(0.25, 4.0, args.tts_train_runs)))
    rng2 = np.random.default_rng(20071102)
    held = list(zip(rng2.uniform(0.25, 2.5, args.tts_eval), rng2.uniform(0.25, 4.0, args.tts_eval)))
    t0 = time.perf_counter()
    x, t, its = warmstart.collect(train, (-5.0, 10.0, 0.1, 10.0, 0.1), 32, "mixed_bf16", tol=1e-7, max_iter=150)
    t_collect = time.perf_counter() - t0
    t0 = time.perf_counter()
    params, losses = warmstart.train(x, t, steps=6000, batch=4096, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    g = api.contour_grid(W["t_min"], W["t_max"], W["dt"], W["beta"], W["dtau"])
    rows = []
    for U, E in held:
        m = api.make_model(float(U), float(E))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        zero = api.dmft_solve(g, m, W["n_quad"], "mixed_bf16", tol=tol, max_iter=150)
        t_zero = time.perf_counter() - t0
        t0 = time.perf_counter()
        s0 = warmstart.warm_start(g, m, params)
        warm = api.dmft_solve(g, m, W["n_quad"], "mixed_bf16", sigma_init=s0, tol=tol, max_iter=150)
        t_warm = time.perf_counter() - t0
        diff = float((warm.gloc - zero.gloc).abs().max() / zero.gloc.abs().max())
        rows.append({"U": float(U), "E": float(E), "iters_zero": zero.iterations, "iters_warm": warm.iterations,
                     "s_zero": t_zero, "s_warm": t_warm, "gloc_rel_diff": diff,
                     "converged": bool(zero.converged and warm.converged)})
    # FP64: one lattice step and one impurity step, timed
    m = api.make_model(float(held[0][0]), float(held[0][1]))
    eps, ebar, wq = api.quadrature_grid(W["n_quad"])
    sig = torch.zeros((g.n_c, g.n_c), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gl, _, _ = api.lattice_gloc(g, m, sig, eps, ebar, wq, precision="fp64")
    torch.cuda.synchronize()
    t_lat64 = time.perf_counter() - t0
    t0 = time.perf_counter()
    api.impurity_update(g, m, gl, sig)
    torch.cuda.synchronize()
    t_imp = time.perf_counter() - t0
    it_zero = np.mean([r["iters_zero"] for r in rows])
    line = {"experiment": "time_to_solution", "tol": tol, "config": W["name"],
            "train": {"runs": len(train), "n_c": 400, "points": 1024, "collect_s": t_collect, "train_s": t_train,
                      "loss_start": float(losses[:20].mean()), "loss_end": float(losses[-100:].mean()),
                      "iters_per_run": its},
            "runs": rows,
            "mixed_zero_s": float(np.mean([r["s_zero"] for r in rows])),
            "mixed_warm_s": float(np.mean([r["s_warm"] for r in rows])),
            "fp64_iteration_s": t_lat64 + t_imp, "fp64_impurity_s": t_imp,
            "fp64_s_estimated": (t_lat64 + t_imp) * it_zero,
            "note": "fp64_s_estimated = measured FP64 lattice + impurity step x mean zero-start iterations"}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.tts:
        run_tts(args)
        return

    import torch

    from paper_0711_0999_gb300 import _native as N
    from paper_0711_0999_gb300 import api, sharding
    from paper_0711_0999_gb300.synth import workload_sigma

    # the oracle pool starts before the first GPU call
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample = oracle_sample(args.cpu_points or None)
        cpu = {"value": v, "unit": "iterations/s", "cores": cores, "kind": "oracle", "sample": sample}

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    W = dict(WORKLOAD)
    if args.n_quad:
        W["n_quad"] = args.n_quad
        W["name"] += f" [profiling subset: {args.n_quad}x{args.n_quad} points]"
    grid = api.contour_grid(W["t_min"], W["t_max"], W["dt"], W["beta"], W["dtau"])
    # independent run per rank (weak scaling): rank r solves U + 0.05 r
    U = W["U"] + 0.05 * rank
    model = api.make_model(U, W["E"])
    eps, ebar, wq = api.quadrature_grid(W["n_quad"])
    nq = len(eps)
    sigma_h = workload_sigma(grid.t, grid.w, U)
    sigma = torch.as_tensor(sigma_h, device=dev)
    eps_d = torch.as_tensor(eps, device=dev)
    ebar_d = torch.as_tensor(ebar, device=dev)
    wq_d = torch.as_tensor(wq, device=dev)
    prec = args.precision
    ws = api.workspace(api.lattice_workspace_size(grid, nq, prec), dev)
    gloc = torch.empty((grid.n_c, grid.n_c), dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        api.lattice_gloc(grid, model, sigma, eps_d, ebar_d, wq_d, precision=prec, ws=ws, out=gloc, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    api.check_status()

    clocks = ClockSampler(local)
    lib = N.lib()
    barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    lib.nedmft_instrument(1, 1)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms = ev0.elapsed_time(ev1)
    launches = N.ctypes.c_int64(0)
    timed = N.ctypes.c_int64(0)
    tms = N.c_double(0.0)
    tfl = N.c_double(0.0)
    tby = N.c_double(0.0)
    lib.nedmft_instrument_read(N.ctypes.byref(launches), N.ctypes.byref(timed), N.ctypes.byref(tms),
                               N.ctypes.byref(tfl), N.ctypes.byref(tby))
    lib.nedmft_instrument(0, 0)
    clk = clocks.stop()
    api.check_status()
    ms = sharding.max_over_ranks(ms, dev)  # the job's time is its slowest rank's
    ms_per_step = ms / args.steps
    value = world * args.steps / (ms / 1e3)
    n = grid.n_c
    flops_bform = 8.0 * n ** 3 * nq
    tflops_step = flops_bform / (ms_per_step / 1e3) / 1e12
    kern_tflops = (tfl.value / (tms.value / 1e3) / 1e12) if tms.value > 0 else 0.0
    kern_gbs = (tby.value / (tms.value / 1e3) / 1e9) if tms.value > 0 else 0.0

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        sig_h = torch.as_tensor(sigma_h).pin_memory()
        e_h, b_h, w_h = (torch.as_tensor(a).pin_memory() for a in (eps, ebar, wq))
        g_h = torch.empty((n, n), dtype=torch.complex128).pin_memory()
        j_h = torch.empty(grid.n_t, dtype=torch.float64).pin_memory()
        ji_h = torch.empty(grid.n_t, dtype=torch.float64).pin_memory()
        sig_d2, e_d2, b_d2, w_d2 = (torch.empty_like(x, device=dev) for x in (sig_h, e_h, b_h, w_h))

        def e2e_step():
            for d, h in ((sig_d2, sig_h), (e_d2, e_h), (b_d2, b_h), (w_d2, w_h)):
                d.copy_(h, non_blocking=True)
            gl, j, ji = api.lattice_gloc(grid, model, sig_d2, e_d2, b_d2, w_d2, precision=prec, ws=ws, out=gloc,
                                         stream=stream)
            g_h.copy_(gl, non_blocking=True)
            j_h.copy_(j, non_blocking=True)
            ji_h.copy_(ji, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize(dev)
        barrier()
        e_s = sharding.max_over_ranks(time.perf_counter() - t0, dev)
        h2d = sig_h.numel() * 16 + 3 * nq * 8
        d2h = g_h.numel() * 16 + 2 * grid.n_t * 8
        e2e = {"value": world * args.steps / e_s, "unit": "iterations/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # one impurity step on the same stream (not part of the timed lattice step)
    ev2 = torch.cuda.Event(enable_timing=True)
    ev3 = torch.cuda.Event(enable_timing=True)
    ws_imp = api.workspace(N.lib().nedmft_impurity_workspace_size(N.ctypes.byref(grid.contour)), dev)
    ev2.record(stream)
    api.impurity_update(grid, model, gloc, sigma, ws=ws_imp, stream=stream)
    ev3.record(stream)
    torch.cuda.synchronize(dev)
    imp_ms = ev2.elapsed_time(ev3)

    peaks, src = load_peaks()
    roof = roofline_for(prec, kern_tflops, kern_gbs, peaks, src, clk)
    roof["kernel"] = "Gauss-Jordan trailing update"
    roof["launches_timed"] = int(timed.value)
    roof["ms_per_launch"] = tms.value / max(1, int(timed.value))
    roof["share_of_step"] = tms.value / ms if ms > 0 else None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "iterations/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": DTYPES[prec], "data": "synthetic",
                "config": {"workload": W["name"], "n_c": n, "points": nq, "precision": prec,
                           "step": "one lattice step: B_q - S build, 2809 Dyson solves, FP64 G_loc and j(t) sums",
                           "parallelism": f"dp{world} (one independent run per GPU)",
                           "l2": "inputs larger than L2 (every step streams >1 GB)"},
                "tflops": tflops_step, "tflops_basis": "B-form 8 N_c^3 per solve",
                "solves_per_s": value * nq,
                "impurity_ms": imp_ms, "dmft_iteration_ms": ms_per_step + imp_ms,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches.value),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
