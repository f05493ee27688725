#!/usr/bin/env python3
"""Benchmark of the nonequilibrium-DMFT solver on GB300.

One step = one DMFT iteration of the N_c = 1500 production configuration
(U = E = 1, beta = 10, t in [-5, 30], dt = 0.05, dtau = 0.1, 53 x 53
Gauss-Hermite points = 2809 solves) with a fixed synthetic self-energy: the
lattice step (every hot-path row: the closed-form B_q - S generation, the
Dyson solve of every quadrature point, the FP64 sums of G_loc and j(t)) and
the impurity step that turns G_loc into the next self-energy.  Prints one
JSON line (rank 0) with the device-timed rate, an end-to-end rate through the
public calls with host buffers, the roofline of the dominant kernel, the
oracle timed on the host cores, the time to a converged solution (mixed path
from zero, mixed path from the learned warm start, FP64 path) and the error
of each output against the FP64 path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores
  python bench.py --tts                  # the full warm-start study (16 held-out pairs)
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="production N_c=1500 (U=1, E=1, beta=10, t in [-5,30], dt=0.05, dtau=0.1, 53x53 points)",
                t_min=-5.0, t_max=30.0, dt=0.05, beta=10.0, dtau=0.1, U=1.0, E=1.0, n_quad=53)
# the warm-start configuration: training runs on a shorter contour, evaluation on the production one
# (the network learns the discrete impurity Green's function at two steps, dt = 0.1 and 0.2, and the warm
# start extrapolates in dt to the production step 0.05)
WARM_TRAIN = dict(contours=((-5.0, 10.0, 0.1, 10.0, 0.1), (-5.0, 10.0, 0.2, 10.0, 0.1)), n_quad=32,
                  U=(0.25, 2.5), E=(0.25, 4.0), seed=20071101)
TTS_TOL = 1e-6  # the paper's pointwise convergence criterion (one part in 10^6)
METRIC = "DMFT iterations/s & TFLOP/s at N_c≈1500; mixed+warm-start vs FP64 at 1e-6 err"
DTYPES = {"fp64": "f64", "mixed_bf16": "bf16x3+f64"}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed_bf16", choices=["fp64", "mixed_bf16"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tts", action="store_true", help="skip the time-to-solution block of the default run")
    ap.add_argument("--cpu-points", type=int, default=0, help="oracle lattice sample per step (0 = automatic)")
    ap.add_argument("--n-quad", type=int, default=0, help="override the quadrature size (profiling runs only)")
    ap.add_argument("--tts", action="store_true", help="the full warm-start study only (16 held-out pairs)")
    ap.add_argument("--tts-train-runs", type=int, default=0, help="training runs (0: 16 default run, 64 --tts)")
    ap.add_argument("--tts-eval", type=int, default=0,
                    help="held-out pairs (0: the first on each side of the Mott transition in the default run, "
                         "16 with --tts)")
    ap.add_argument("--config", default="cfg1", choices=["cfg1", "cfg2", "cfg3"],
                    help="cfg1: the production step (default); cfg2: the ragged sweep of 48 runs with dt -> 0 "
                         "extrapolation; cfg3: one step of the N_c = 3400 Mott configuration")
    ap.add_argument("--max-iter", type=int, default=40, help="iteration cap of the cfg2 sweep")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ CPU oracle timing


def _oracle_points(task):
    """The oracle's lattice work for a few points: G0 build and solve(I - G0 S, G0)."""
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
    """The oracle, as it stands, on bounded samples of one DMFT iteration of the
    workload, on all host cores: the lattice points on one spawned process pool
    (one BLAS thread per process, the paper's parallel axis) that lives across
    warm-up and timed steps, and the impurity step (serial in the method) in
    this process with the BLAS library's threads on every core."""

    def __init__(self):
        import multiprocessing as mp

        from oracle import nedmft_oracle as O
        from paper_0711_0999_gb300.synth import workload_sigma

        W = WORKLOAD
        self.O = O
        self.cores = os.cpu_count() or 1
        self.c = O.contour_grid(W["t_min"], W["t_max"], W["dt"], W["beta"], W["dtau"])
        self.model = O.Model(U=W["U"], E=W["E"])
        self.sigma = workload_sigma(self.c.t, self.c.w, W["U"])
        # a stand-in for G_loc (the inversions cost the same for any nonsingular matrix)
        self.gloc = -0.5j * np.eye(self.c.n_c) + 0.01 * self.sigma
        self.eps, self.ebar, _ = O.quadrature_points(W["n_quad"])
        self.nq = len(self.eps)
        env = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in env:
            os.environ[k] = "1"  # the spawned workers: one BLAS thread each
        self.pool = mp.get_context("spawn").Pool(processes=self.cores)
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v

    def _tasks(self, npts):
        W = WORKLOAD
        idx = np.linspace(0, self.nq - 1, npts).round().astype(int)
        return [(W["t_min"], W["t_max"], W["dt"], W["beta"], W["dtau"], W["U"], W["E"], self.sigma,
                 [(float(self.eps[i]), float(self.ebar[i]))]) for i in idx]

    def warm(self):
        """One point per process and one impurity step, untimed (start-up, imports, first solves)."""
        self.pool.map(_oracle_points, self._tasks(self.cores))
        self.O.impurity_update(self.c, self.model, self.gloc, self.sigma)

    def time(self, npts: int):
        """DMFT iterations/s from `npts` evenly spread lattice points (scaled to
        all points) plus one impurity step, the cores used and a description."""
        tasks = self._tasks(npts)
        t0 = time.perf_counter()
        self.pool.map(_oracle_points, tasks)
        t_lat = (time.perf_counter() - t0) * self.nq / npts
        t0 = time.perf_counter()
        self.O.impurity_update(self.c, self.model, self.gloc, self.sigma)
        t_imp = time.perf_counter() - t0
        sample = (f"{npts} of {self.nq} lattice points of the N_c={self.c.n_c} workload (G0 build + "
                  f"solve(I - G0 S, G0) each) on {min(self.cores, npts)} processes x 1 BLAS thread, scaled by "
                  f"{self.nq}/{npts} to {t_lat:.1f} s, plus one impurity step (4 inversions) in one process "
                  f"with BLAS threads on {self.cores} cores, {t_imp:.1f} s")
        return 1.0 / (t_lat + t_imp), self.cores, sample

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_sample(n_points: int | None = None):
    """One timed sample (default 5 lattice points per host core) after one
    warm-up round: (DMFT iterations/s, cores, sample text)."""
    t = OracleTimer()
    try:
        t.warm()
        return t.time(n_points or 5 * t.cores)
    finally:
        t.close()


def reference_points_per_step(cores: int, steps: int) -> int:
    """Lattice points per timed step of the reference arm: a multiple of the
    core count (so no process idles in the last round), 5 per core for up to
    5 steps, then fewer, never under one per core, so that K steps together
    stay at about 25 points per core whatever K is."""
    return cores * max(1, 25 // max(steps, 5))


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


# ------------------------------------------------------------------ peaks and roofline


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


# DRAM bytes of one Gauss-Jordan update launch (152 matrices at N_c = 1500) from
# an ncu capture of the kernel as it stands; None while the kernel has changed
# since the counters were taken
UPDATE_TRAFFIC_BYTES = 6.33e9
UPDATE_TRAFFIC_NOTE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on 16 matrices "
                       "(396.8 + 269.1 MB), scaled by 152/16 to the 152-matrix launch; 1.10x the "
                       "algorithmic 2 x N_c^2 x 8 B per matrix: the rest is the C' and R operand panels")


def roofline_for(precision: str, tflops: float, gbs: float, peaks, src: str):
    """Roofline of the dominant kernel from its algorithmic rate.

    Mixed path: the Gauss-Jordan trailing update, a dense contraction whose
    algorithmic work is 8 N_c^2 W real flops per matrix per rank-W step (the
    complex multiply-add counted as 8).  It runs as bf16 tensor-core products,
    so the peak is the measured dense bf16 rate (the sustained figure: the
    kernel runs inside a long step) and `frac` is the method's flops over it.
    Every algorithmic flop costs three bf16 products (bf16x3), so the tensor
    pipe is busy about 3 x frac of the time: `tensor_pipe_frac`.
    FP64 path: FP64 arithmetic on CUDA cores against the part's nominal rate."""
    if precision == "mixed_bf16":
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        hpeak = peaks["hbm_gbs"]
        return {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                "traffic": UPDATE_TRAFFIC_BYTES, "traffic_note": UPDATE_TRAFFIC_NOTE,
                "peak_source": f"sustained dense bf16 tensor rate, {src}",
                "tensor_pipe_frac": 3.0 * tflops / peak,
                "tensor_pipe_note": "bf16x3: three bf16 products (hi*hi, hi*lo, lo*hi) per algorithmic flop",
                "hbm": {"achieved": gbs, "peak": hpeak, "unit": "GB/s", "frac": gbs / hpeak,
                        "note": "algorithmic read + write of the FP32 complex matrix per step"}}
    peak = 1.25  # nominal FP64 rate of the part
    return {"bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
            "traffic": None, "peak_source": "nominal FP64 1.25 TFLOP/s", "hbm_gbs": gbs}


# ------------------------------------------------------------------ reference arm


def run_reference(args, rank, world):
    if rank != 0:
        return
    rates = []
    cores = sample = None
    t = OracleTimer()
    try:
        for _ in range(max(args.warmup, 1)):
            t.warm()
        npts = args.cpu_points or reference_points_per_step(t.cores, args.steps)
        for _ in range(args.steps):
            v, cores, sample = t.time(npts)
            rates.append(v)
    finally:
        t.close()
    v = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "iterations/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "n_c": 1500, "points": WORKLOAD["n_quad"] ** 2,
                       "step": "one DMFT iteration (lattice step + impurity step)",
                       "parallelism": "host process pool"},
            "cpu_baseline": {"value": v, "unit": "iterations/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ time to solution


def warm_start_network(n_runs: int, log=None):
    """Train the warm-start network on converged plain solves of `n_runs` (U, E)
    pairs drawn like the warm-start configuration; returns (params, info)."""
    import torch

    from paper_0711_0999_gb300 import warmstart

    rng = np.random.default_rng(WARM_TRAIN["seed"])
    runs = list(zip(rng.uniform(*WARM_TRAIN["U"], n_runs), rng.uniform(*WARM_TRAIN["E"], n_runs)))
    t0 = time.perf_counter()
    x, t, its, conv = warmstart.collect(runs, WARM_TRAIN["contours"], WARM_TRAIN["n_quad"], "mixed_bf16", tol=1e-7,
                                        max_iter=150)
    torch.cuda.synchronize()
    t_collect = time.perf_counter() - t0
    t0 = time.perf_counter()
    params, losses = warmstart.train(x, t, steps=6000, batch=4096, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    losses = losses.cpu().numpy()
    return params, {"runs": n_runs, "solves": len(conv), "solves_converged": int(sum(conv)), "n_c": [400, 250],
                    "dt": [0.1, 0.2],
                    "points": WARM_TRAIN["n_quad"] ** 2, "collect_s": t_collect,
                    "train_s": t_train, "loss_start": float(losses[:20].mean()),
                    "loss_end": float(losses[-100:].mean()), "iterations_per_run": its}


def held_out_pairs(n: int):
    rng = np.random.default_rng(WARM_TRAIN["seed"] + 1)
    return list(zip(rng.uniform(*WARM_TRAIN["U"], n), rng.uniform(*WARM_TRAIN["E"], n)))


def default_held_out_pairs(u_mott: float):
    """The first pair of the 16 held-out ones on each side of the Mott
    transition (insulating first: the warm start is gated off there, so that
    pair measures the plain loop, the metallic one the warm start)."""
    pairs = held_out_pairs(16)
    return [next(p for p in pairs if p[0] >= u_mott), next(p for p in pairs if p[0] < u_mott)]


def time_to_solution(n_train: int, n_eval: int, with_fp64: bool = True, pairs=None):
    """Converged DMFT at N_c = 1500 to the paper's pointwise criterion (1e-6):
    the mixed path from Sigma = 0, from the closed-form band alone and from the
    learned warm start; the FP64 path's iteration (lattice + impurity step,
    measured) times the zero-start iteration count; and the error of each
    output (G_loc, j, Sigma after one impurity step) of the mixed path against
    the FP64 path at the converged self-energy of the first pair."""
    import torch

    from paper_0711_0999_gb300 import api, warmstart

    W = WORKLOAD
    out = {"tol": TTS_TOL, "config": W["name"]}
    params = None
    if n_train > 0:
        params, out["train"] = warm_start_network(n_train)
    g = api.contour_grid(W["t_min"], W["t_max"], W["dt"], W["beta"], W["dtau"])
    rows = []
    first = None

    def solve(model, init):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s0 = init() if init is not None else None
        sol = api.dmft_solve(g, model, W["n_quad"], "mixed_bf16", sigma_init=s0, tol=TTS_TOL, max_iter=150)
        torch.cuda.synchronize()
        return sol, time.perf_counter() - t0

    for U, E in (pairs if pairs is not None else held_out_pairs(n_eval)):
        m = api.make_model(float(U), float(E))
        zero, t_zero = solve(m, None)
        band, t_band = solve(m, lambda: warmstart.band_only(g, m))
        row = {"U": float(U), "E": float(E), "iters_zero": zero.iterations, "s_zero": t_zero,
               "iters_band": band.iterations, "s_band": t_band, "converged": bool(zero.converged)}
        if params is not None:
            warm, t_warm = solve(m, lambda: warmstart.initial_sigma(g, m, params))
            row.update({"iters_warm": warm.iterations, "s_warm": t_warm, "converged": bool(row["converged"] and
                                                                                            warm.converged),
                        "gloc_rel_diff_warm_vs_zero": float((warm.gloc - zero.gloc).abs().max() /
                                                            zero.gloc.abs().max())})
        rows.append(row)
        if first is None:
            first = (m, zero)
    out["runs"] = rows
    mean = lambda k: float(np.mean([r[k] for r in rows])) if rows and k in rows[0] else None
    out.update({"mixed_zero_s": mean("s_zero"), "mixed_band_s": mean("s_band"), "mixed_warm_s": mean("s_warm"),
                "iters_zero": mean("iters_zero"), "iters_band": mean("iters_band"), "iters_warm": mean("iters_warm")})
    if with_fp64 and first is not None:
        m, zero = first
        eps, ebar, wq = api.quadrature_grid(W["n_quad"])
        dev = zero.sigma.device
        e_d, b_d, w_d = (torch.as_tensor(a, device=dev) for a in (eps, ebar, wq))
        sig = zero.sigma
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g64, j64, _ = api.lattice_gloc(g, m, sig, e_d, b_d, w_d, precision="fp64")
        torch.cuda.synchronize()
        t_lat = time.perf_counter() - t0
        t0 = time.perf_counter()
        s64, _ = api.impurity_update(g, m, g64, sig)
        torch.cuda.synchronize()
        t_imp = time.perf_counter() - t0
        gmx, jmx, _ = api.lattice_gloc(g, m, sig, e_d, b_d, w_d, precision="mixed_bf16")
        smx, _ = api.impurity_update(g, m, gmx, sig)
        torch.cuda.synchronize()
        api.check_status()
        w = torch.as_tensor(g.w, device=dev)
        ws = lambda s: w[:, None] * s * w[None, :]  # W Sigma W, the operator the solve uses
        fp64_total = float(np.mean([(t_lat + t_imp) * r["iters_zero"] for r in rows]))
        out["fp64"] = {"lattice_s": t_lat, "impurity_s": t_imp, "iteration_s": t_lat + t_imp,
                       "total_s_extrapolated": fp64_total,
                       "note": "FP64 lattice + impurity step measured at the converged Sigma of the first pair, "
                               "times each pair's zero-start iteration count of the mixed path, averaged over "
                               "the pairs (not run to convergence)"}
        out["errors_vs_fp64"] = {
            "gloc_rel": float((gmx - g64).abs().max() / g64.abs().max()),
            "j_abs": float((jmx - j64).abs().max()),
            "sigma_next_rel": float((ws(smx) - ws(s64)).abs().max() / ws(s64).abs().max()),
            "where": "one lattice + impurity step at the converged mixed-path Sigma of the first pair; the FP64 "
                     "path itself matches the oracle to 3e-14 at this configuration (full-grid test)"}
        if out["mixed_zero_s"]:
            out["speedup_mixed_zero_vs_fp64"] = out["fp64"]["total_s_extrapolated"] / out["mixed_zero_s"]
        if out["mixed_warm_s"]:
            out["speedup_mixed_warm_vs_fp64"] = out["fp64"]["total_s_extrapolated"] / out["mixed_warm_s"]
    return out


# ------------------------------------------------------------------ other configurations


CFG2 = dict(U=(0.5, 1.0, 1.5, 2.0), E=(0.5, 1.0, 2.0, 4.0), dts=(0.1, 1.0 / 15.0, 0.05), t_min=-5.0, t_max=25.0,
            beta=10.0, dtau=0.1, n_quad=40)
CFG3 = dict(t_min=-5.0, t_max=50.0, dt=1.0 / 30.0, beta=10.0, dtau=0.1, U=2.0, E=1.0, n_quad=64)


def run_cfg2(args):
    """The ragged sweep: U in {0.5, 1, 1.5, 2} x E in {0.5, 1, 2, 4} x dt in
    {0.1, 1/15, 0.05} (N_c = 700 / 1000 / 1300), t in [-5, 25], beta = 10,
    40 x 40 points, all 48 runs swept together (one iteration of every active
    run per host synchronisation) to 1e-6 or the iteration cap, then the
    quadratic dt -> 0 Lagrange extrapolation of every (U, E)'s current in FP64."""
    import torch

    from paper_0711_0999_gb300 import api

    torch.cuda.set_device(0)
    C = CFG2
    pairs = [(U, E) for U in C["U"] for E in C["E"]]
    grids = {dt: api.contour_grid(C["t_min"], C["t_max"], dt, C["beta"], C["dtau"]) for dt in C["dts"]}
    runs = [(U, E, dt) for U, E in pairs for dt in C["dts"]]
    gl = [grids[dt] for _, _, dt in runs]
    models = [api.make_model(U, E) for U, E, _ in runs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sols = api.dmft_solve_batch(gl, models, C["n_quad"], args.precision, tol=TTS_TOL, max_iter=args.max_iter)
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    t_out = np.arange(C["t_min"], C["t_max"] - 0.2 + 1e-9, 0.2)  # times on all three grids
    t0 = time.perf_counter()
    extrap = []
    for k, (U, E) in enumerate(pairs):
        cur = [sols[3 * k + r].current for r in range(3)]
        extrap.append(api.extrapolate_current([grids[dt] for dt in C["dts"]], cur, t_out))
    torch.cuda.synchronize()
    t_extrap = time.perf_counter() - t0
    nq = C["n_quad"] ** 2
    flops = sum(s.iterations * 8.0 * g.n_c ** 3 * nq for s, g in zip(sols, gl))  # B-form, lattice steps only
    its = [s.iterations for s in sols]
    line = {"experiment": "cfg2 ragged sweep", "precision": args.precision, "runs": len(runs),
            "converged": int(sum(s.converged for s in sols)), "iterations": its, "iteration_cap": args.max_iter,
            "lattice_steps": int(sum(its)), "solve_s": t_solve, "runs_per_s": len(runs) / t_solve,
            "lattice_steps_per_s": sum(its) / t_solve, "tflops_lattice_bform": flops / t_solve / 1e12,
            "extrapolation_s": t_extrap, "extrapolated_pairs": len(pairs),
            "j_extrapolated_max_abs": [float(e.abs().max()) for e in extrap],
            "n_c": sorted({g.n_c for g in gl}), "points": nq,
            "note": "dmft_solve_batch: one iteration of every active run per host sync; each run's points fill "
                    "its own Gauss-Jordan batches"}
    print(json.dumps(line), flush=True)


def run_cfg3(args):
    """One DMFT iteration (lattice + impurity step) of the long Mott contour:
    U = 2, E = 1, t in [-5, 50], dt = 1/30 (N_c = 3400), 64 x 64 points,
    streamed through the Gauss-Jordan in batches sized to HBM, with the
    synthetic self-energy workload; one untimed iteration first."""
    import torch

    from paper_0711_0999_gb300 import _native as N
    from paper_0711_0999_gb300 import api
    from paper_0711_0999_gb300.synth import workload_sigma

    torch.cuda.set_device(0)
    C = CFG3
    g = api.contour_grid(C["t_min"], C["t_max"], C["dt"], C["beta"], C["dtau"])
    m = api.make_model(C["U"], C["E"])
    eps, ebar, wq = api.quadrature_grid(C["n_quad"])
    dev = torch.device("cuda")
    sig = torch.as_tensor(workload_sigma(g.t, g.w, C["U"]), device=dev)
    e_d, b_d, w_d = (torch.as_tensor(a, device=dev) for a in (eps, ebar, wq))
    ws = api.workspace(api.lattice_workspace_size(g, len(wq), args.precision), dev)
    ws_imp = api.workspace(N.lib().nedmft_impurity_workspace_size(N.ctypes.byref(g.contour)), dev)
    out = torch.empty((g.n_c, g.n_c), dtype=torch.complex128, device=dev)
    st = torch.cuda.current_stream()

    def iteration():
        api.lattice_gloc(g, m, sig, e_d, b_d, w_d, precision=args.precision, ws=ws, out=out, stream=st)
        ev[1].record(st)
        api.impurity_update(g, m, out, sig, ws=ws_imp, stream=st)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    iteration()
    torch.cuda.synchronize()
    ev[0].record(st)
    iteration()
    ev[2].record(st)
    torch.cuda.synchronize()
    api.check_status()
    lat = ev[0].elapsed_time(ev[1]) / 1e3
    imp = ev[1].elapsed_time(ev[2]) / 1e3
    nq = len(wq)
    line = {"experiment": "cfg3 long contour", "precision": args.precision, "n_c": g.n_c, "points": nq,
            "points_per_batch": api.lattice_batch(g, nq, args.precision), "lattice_s": lat, "impurity_s": imp,
            "iteration_s": lat + imp, "solves_per_s": nq / lat,
            "tflops_lattice_bform": 8.0 * g.n_c ** 3 * nq / lat / 1e12,
            "workspace_gb": ws.numel() / 1e9}
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
    if args.config == "cfg2":
        run_cfg2(args)
        return
    if args.config == "cfg3":
        run_cfg3(args)
        return
    if args.tts:
        import torch
        torch.cuda.set_device(0)
        line = {"experiment": "time_to_solution"}
        line.update(time_to_solution(args.tts_train_runs or 64, args.tts_eval or 16))
        print(json.dumps(line), flush=True)
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
    n = grid.n_c
    ws = api.workspace(api.lattice_workspace_size(grid, nq, prec), dev)
    ws_imp = api.workspace(N.lib().nedmft_impurity_workspace_size(N.ctypes.byref(grid.contour)), dev)
    gloc = torch.empty((n, n), dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream(dev)

    def iteration():
        """One DMFT iteration: lattice step on Sigma, impurity step on its G_loc."""
        api.lattice_gloc(grid, model, sigma, eps_d, ebar_d, wq_d, precision=prec, ws=ws, out=gloc, stream=stream)
        ev_mid.append(torch.cuda.Event(enable_timing=True))
        ev_mid[-1].record(stream)
        api.impurity_update(grid, model, gloc, sigma, ws=ws_imp, stream=stream)

    ev_mid = []
    for _ in range(args.warmup):
        iteration()
    torch.cuda.synchronize(dev)
    api.check_status()

    clocks = ClockSampler(local)
    lib = N.lib()
    barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    lib.nedmft_instrument(1, 1)
    ev_start = []
    ev_mid = []
    ev_end = []
    for _ in range(args.steps):
        ev_start.append(torch.cuda.Event(enable_timing=True))
        ev_start[-1].record(stream)
        iteration()
        ev_end.append(torch.cuda.Event(enable_timing=True))
        ev_end[-1].record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms = ev_start[0].elapsed_time(ev_end[-1])
    lat_ms = sum(a.elapsed_time(b) for a, b in zip(ev_start, ev_mid))
    imp_ms = sum(a.elapsed_time(b) for a, b in zip(ev_mid, ev_end))
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
    lat_step_ms = lat_ms / args.steps
    imp_step_ms = imp_ms / args.steps
    flops_lattice = 8.0 * n ** 3 * nq            # B-form: one complex inversion per point
    flops_impurity = 2 * 8.0 * n ** 3            # two complex inversions
    kern_tflops = (tfl.value / (tms.value / 1e3) / 1e12) if tms.value > 0 else 0.0
    kern_gbs = (tby.value / (tms.value / 1e3) / 1e9) if tms.value > 0 else 0.0

    # end to end through the public calls with host buffers: every step copies
    # its inputs from pinned host memory, runs the lattice and impurity steps
    # and reads G_loc, the current and the new self-energy back
    e2e = None
    if not args.no_e2e:
        sig_h = torch.as_tensor(sigma_h).pin_memory()
        e_h, b_h, w_h = (torch.as_tensor(a).pin_memory() for a in (eps, ebar, wq))
        g_h = torch.empty((n, n), dtype=torch.complex128).pin_memory()
        s_h = torch.empty((n, n), dtype=torch.complex128).pin_memory()
        j_h = torch.empty(grid.n_t, dtype=torch.float64).pin_memory()
        sig_d2, e_d2, b_d2, w_d2 = (torch.empty_like(x, device=dev) for x in (sig_h, e_h, b_h, w_h))

        def e2e_step():
            for d, h in ((sig_d2, sig_h), (e_d2, e_h), (b_d2, b_h), (w_d2, w_h)):
                d.copy_(h, non_blocking=True)
            gl, j, _ = api.lattice_gloc(grid, model, sig_d2, e_d2, b_d2, w_d2, precision=prec, ws=ws, out=gloc,
                                        stream=stream)
            s_new, _ = api.impurity_update(grid, model, gl, sig_d2, ws=ws_imp, stream=stream)
            g_h.copy_(gl, non_blocking=True)
            s_h.copy_(s_new, non_blocking=True)
            j_h.copy_(j, non_blocking=True)

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
        d2h = g_h.numel() * 16 + s_h.numel() * 16 + grid.n_t * 8
        e2e = {"value": world * args.steps / e_s, "unit": "iterations/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "calls": "nedmft_lattice_gloc + nedmft_impurity_update per step"}

    tts = None
    if rank == 0 and world == 1 and not args.no_tts and not args.n_quad:
        from paper_0711_0999_gb300 import warmstart

        tts = time_to_solution(args.tts_train_runs or 16, args.tts_eval,
                               pairs=None if args.tts_eval else default_held_out_pairs(warmstart.U_MOTT))

    peaks, src = load_peaks()
    roof = roofline_for(prec, kern_tflops, kern_gbs, peaks, src)
    roof["kernel"] = "Gauss-Jordan trailing update" if prec == "mixed_bf16" else "FP64 Gauss-Jordan update"
    roof["launches_timed"] = int(timed.value)
    roof["ms_per_launch"] = tms.value / max(1, int(timed.value))
    roof["share_of_step"] = tms.value / ms if ms > 0 else None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "iterations/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": DTYPES[prec], "data": "synthetic",
                "config": {"workload": W["name"], "n_c": n, "points": nq, "precision": prec,
                           "step": "one DMFT iteration: lattice step (B_q - S build, 2809 Dyson solves, FP64 "
                                   "G_loc and j(t) sums) + impurity step (2 FP64 inversions)",
                           "parallelism": f"dp{world} (one independent run per GPU)",
                           "l2": "inputs larger than L2 (every step streams >1 GB)"},
                "lattice_ms": lat_step_ms, "impurity_ms": imp_step_ms, "lattice_steps_per_s": 1e3 / lat_step_ms,
                "tflops": (flops_lattice + flops_impurity) / (ms_per_step / 1e3) / 1e12,
                "tflops_lattice": flops_lattice / (lat_step_ms / 1e3) / 1e12,
                "tflops_basis": "B-form 8 N_c^3 per solve; impurity 2 x 8 N_c^3 (two inversions)",
                "solves_per_s": nq / (lat_step_ms / 1e3),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches.value),
                "clocks": clk, "tts": tts}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
