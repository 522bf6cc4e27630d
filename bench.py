#!/usr/bin/env python
"""Time-to-solution per time step of MLGMRES on the 256^2 moving-Gaussian
Poisson series (GMRES(30), relative residual 1e-10): the learned initial guess
with FP32-inner / FP64-refined GMRES, next to plain FP64 GMRES from x0 = 0 and
from x0 = x_{t-1}, the same solver without the network, and a smoothing-only
control, all on the same GPU, plus the FP64 CPU oracle on the host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  A "step" is one time step of the online loop:
the network's guess, the solve, Algorithm 1's gate and replay store, and every
10th step the start of a training phase.  Phases run on a low-priority side
stream beside the solves, which run on a high-priority stream and take a
phase's parameters once it has completed; a phase that is still running when
the next one is due holds the loop until it ends, so that time lands in the
step.  Before the W warm-up steps the loop runs its tau0 = 50 online warm-up
steps (data collection and the first training, Sec. 2.3) untimed.

The same line carries, as sub-objects, the other workloads on one GPU: a
capped 2048^2 solve for the HBM roofline (`roofline_hbm`), full time steps of
the 2048^2 refinement workload with the error against the DST-I solution
(`c3_full_steps`, --c3-steps, 1 by default), the 512-instance batched
workload in one persistent launch (`c4_batch`, --no-batch to skip), a capped
192^3 variable-kappa solve (`roofline_3d`) and full time steps of that
workload certified by the true FP64 residual (`c5_full_steps`, --c5-steps, 1
by default).
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE = 256
M = 30
RTOL = 1e-10
T_SERIES = 500
SEED = 2001
TAU0 = 50
TRAIN_EVERY = 10
# training phase and guess post-processing of the learned arms: 64 Adam steps
# (lr 2e-3, minibatch 8) per phase and 32 damped-Jacobi sweeps on the guess.
# Measured on this series: with 32 steps (lr 1e-3) and 8 sweeps the network's
# guess never beats x0 = 0 after one GMRES(30) cycle; with these it does on 80%
# of the steps and saves 13% of the iterations.
LEARN = dict(train_iters=64, lr=2e-3, batch=8, guess_smooth=32, overlap_train=1)
METRIC = "time-to-solution per time step (ms) and GMRES iters, learned vs plain GMRES, rel res 1e-10"
# DRAM bytes per Arnoldi step of gmres_persistent<float, 2, 32, 256, shared V>
# on this workload, from one ncu capture of a 300-step solve of the kernel
# (dram__bytes_read.sum + dram__bytes_write.sum = 1.191 MB + 0.022 MB); scaled
# to a launch by its steps.
DRAM_BYTES_PER_STEP = 1.213e6 / 300
# the same for the compact bulk-copy variant at 2048^2, GMRES(40) (304 CTAs, two
# stages): 58.91 GB + 5.31 GB over an 80-step (two-cycle) capture
DRAM_BYTES_PER_STEP_2048 = 64.22e9 / 80
# and for the 192^3 variable-kappa kernel, GMRES(50), in the shape the autotuner
# picks (the compact variant, 304 CTAs, two stages): 172.99 GB + 11.53 GB over a
# 100-step (two-cycle) capture
DRAM_BYTES_PER_STEP_3D = 184.52e9 / 100
WORKLOAD = ("2D Poisson -Lap u = f, 256x256 interior (N=65,536), zero Dirichlet, 5-point; "
            "3 moving signed Gaussians (sigma 0.1), 500-step series seed 2001; GMRES(30) "
            "rel tol 1e-10 (true FP64 residual)")
# the HBM-bound case: the 2048^2 random-walk workload (16 Gaussians plus a
# sin*sin eigenmode), GMRES(40) FP32 cycles, one solve capped at HBM_STEPS
# Arnoldi steps from x0 = 0
HBM_N, HBM_M, HBM_STEPS = 2048, 40, 400
SMOOTH = 32      # damped-Jacobi sweeps of the learned guess (and of the smoothing-only arm)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-GMRES arms")
    ap.add_argument("--no-hbm", action="store_true", help="skip the 2048^2 roofline solve")
    ap.add_argument("--c3-steps", type=int, default=1,
                    help="full time steps of the 2048^2 workload to time (0 = none; single GPU)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 512-instance batched workload (single GPU)")
    ap.add_argument("--c5-steps", type=int, default=1,
                    help="full time steps of the 192^3 variable-kappa workload to time "
                         "(0 = none; 35-45 s each; single GPU)")
    ap.add_argument("--grid-blocks", type=int, default=0,
                    help="CTAs of the headline solver (0 = autotuned); fixes its launch "
                         "shape, e.g. for a profiler run whose timings would steer the autotuner")
    return ap.parse_args()


# --------------------------------------------------------------- clocks --
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- helpers --
def max_over_ranks(value, dist, device=None):
    """The largest `value` over all ranks (the job's time is its slowest rank's);
    the value itself when not distributed."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_ms_per_step(total_ms_this_rank, steps, world, dist, device=None):
    """Replicas: every rank runs its own series of `steps` time steps; the job
    processed steps * world time steps in the slowest rank's time."""
    return max_over_ranks(total_ms_this_rank, dist, device) / (steps * world)

def _cycles(res, m):
    """Arnoldi steps of each restart cycle of a solve."""
    iters, cycles = int(res["iters"]), int(res["cycles"])
    ncyc = max(cycles, 1 if iters else 0)
    out, left = [], iters
    for c in range(ncyc):
        k = min(m, left) if c < ncyc - 1 else left
        left -= k
        out.append(k)
    return out


def algorithmic_bytes(res, N, m, elem, kappa=False):
    """Bytes a solve must move by the roofline's definition: per Arnoldi step
    j a three-sweep CGS2 with lazy normalisation, elem*N*(3(j+1) + 7) (SpMV
    reads v_j and writes w; the sweeps read V_0..V_j three times, read w three
    times and write it twice); per cycle of k steps x += V y, (k*elem + 16)*N,
    and the FP64 true residual, 32 N."""
    total = 0.0
    for k in _cycles(res, m):
        total += elem * N * (3.0 * k * (k + 1) / 2.0 + 7.0 * k)   # sum_{j<k} 3(j+1) + 7
        if kappa:
            total += 4.0 * N * k                                   # 3D: cell kappa once a step
        total += (k * elem + 16.0) * N + 32.0 * N
    return total


def two_pass_bytes(res, N, m, elem):
    """What this library's two-pass CGS2 step moves: per Arnoldi step j the
    passes read V_0..V_{j-1} and V_0..V_j, w' and z and write v_j, z and w':
    elem*N*(2j + 6); per cycle with k steps x += V y reads k basis vectors and
    x (16 N with its write), and the FP64 restart reads x and b (16 N) and
    writes w'_0 (elem*N)."""
    total = 0.0
    for k in _cycles(res, m):
        total += elem * N * (k * (k - 1) + 6.0 * k)   # sum_j (2j + 6)
        total += elem * N * k + 16.0 * N              # x += V y
        total += 16.0 * N + elem * N                  # restart
    total += 16.0 * N + elem * N                      # final residual check
    return total


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def host_cpu():
    """nproc and the CPU model of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return os.cpu_count() or 1, model


def oracle_threads(b, n):
    """The oracle's fastest thread count on this host (its OpenMP mode, vector
    operations split over threads), from a 60-iteration sample per count."""
    from oracle import native
    nproc, _ = host_cpu()
    best, best_t = 1, None
    for th in sorted({1, 2, 4, 8, 16, 32, 64, nproc}):
        if th > nproc:
            continue
        t0 = time.perf_counter()
        native.gmres(2, n, b, m=M, rtol=RTOL, max_iters=60, nthreads=th)
        dt = time.perf_counter() - t0
        if best_t is None or dt < best_t:
            best, best_t = th, dt
    return best


def cpu_baseline(b, n, t_index):
    """The FP64 oracle (plain GMRES(30), x0 = 0) on one full time step, on all
    host cores (the oracle's OpenMP mode at its fastest thread count) and on
    one thread."""
    from oracle import native
    native.lib()
    nproc, model = host_cpu()
    th = oracle_threads(b, n)
    t0 = time.perf_counter()
    _, st, _ = native.gmres(2, n, b, m=M, rtol=RTOL, nthreads=th)
    dt = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, st1, _ = native.gmres(2, n, b, m=M, rtol=RTOL, nthreads=1)
    dt1 = time.perf_counter() - t0
    return {"value": dt * 1e3, "unit": "ms per time step", "cores": th, "kind": "oracle",
            "sample": "one full time step (t=%d) of the 256^2 series: FP64 GMRES(30), x0=0, "
                      "rtol 1e-10, %d iterations, %d threads (fastest count of the oracle's "
                      "OpenMP mode on this host)" % (t_index, st["iters"], th),
            "iters": st["iters"], "extrapolated": False, "nproc": nproc, "cpu_model": model,
            "single_thread": {"value": dt1 * 1e3, "unit": "ms per time step", "cores": 1,
                              "iters": st1["iters"]}}


# ------------------------------------------------------------ reference --
def run_reference(args):
    """The FP64 oracle as it stands (plain GMRES(30) from x0 = 0; it has no
    network) on the host cores, on the time steps the GPU arm times: W warm-up
    steps as 600-iteration samples (untimed), then K full solves, each timed."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import native
    from synthetic import MovingGaussians2D
    native.lib()
    gen = MovingGaussians2D(N_SIDE, SEED, T_SERIES)
    nproc, model = host_cpu()
    th = oracle_threads(gen.rhs(TAU0), N_SIDE)
    for t in range(args.warmup):
        native.gmres(2, N_SIDE, gen.rhs(TAU0 + t), m=M, rtol=RTOL, max_iters=600, nthreads=th)
    times, iters = [], []
    for t in range(args.steps):
        b = gen.rhs(TAU0 + args.warmup + t)
        t0 = time.perf_counter()
        _, st, _ = native.gmres(2, N_SIDE, b, m=M, rtol=RTOL, nthreads=th)
        times.append(time.perf_counter() - t0)
        iters.append(st["iters"])
    value = 1e3 * statistics.mean(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ms",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": value, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "guess": "zero (the oracle has no network)",
                   "precision": "fp64"},
        "iters_per_step": statistics.mean(iters),
        "extrapolated": False,
        "cpu_baseline": {"value": value, "unit": "ms per time step", "cores": th,
                         "kind": "oracle", "nproc": nproc, "cpu_model": model,
                         "extrapolated": False,
                         "sample": "each timed step is one full FP64 GMRES(30) solve of time step "
                                   "t = %d + i of the 256^2 series (the GPU arm's timed steps), "
                                   "%d threads; warm-up steps are 600-iteration samples"
                                   % (TAU0 + args.warmup, th)},
        "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ours --
def run_ours(args):
    import numpy as np  # noqa: F401
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import paper_2103_10975_gb300 as pkg
    from synthetic import MovingGaussians2D

    n, N = N_SIDE, N_SIDE * N_SIDE
    # replicas: every rank runs its own independent series
    gen = MovingGaussians2D(n, SEED + rank, T_SERIES)
    K, W = args.steps, args.warmup
    t_end = TAU0 + W + 2 * K + 2
    assert t_end <= T_SERIES
    # the solves run on a high-priority stream, training phases on a
    # low-priority one, so the solver's CTAs are dispatched first
    main = torch.cuda.Stream(priority=-100)
    side = torch.cuda.Stream(priority=0)
    torch.cuda.set_stream(main)
    B = torch.stack([torch.as_tensor(gen.rhs(t)) for t in range(t_end)]).to(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    host_train = [0.0]   # host seconds spent in train_step by the last series

    def run_series(solver, t0, count, learned, timed, results, pre=None, drain=True):
        """Steps t0..t0+count-1; returns per-step device ms (events on the solve
        stream).  A step is the solve plus, every TRAIN_EVERY steps, starting a
        training phase (which waits on the host for a phase still running).
        With `drain`, the time the solve stream then waits for the last phase
        to end is added to the last step, so no training is left uncounted."""
        ms = []
        x = None
        host_train[0] = 0.0
        for i in range(count):
            t = t0 + i
            if timed:
                flush.fill_(float(i))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(main)
            if pre is not None:
                x = pre(solver, B[t])
            x, r = solver.solve(B[t], x)
            if learned and (t + 1) % TRAIN_EVERY == 0:
                h0 = time.perf_counter()
                solver.train_step(stream=side)
                host_train[0] += time.perf_counter() - h0
            e1.record(main)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            results.append(r)
        if learned and drain and count:
            d0 = torch.cuda.Event(enable_timing=True)
            d1 = torch.cuda.Event(enable_timing=True)
            d0.record(main)
            main.wait_stream(side)
            d1.record(main)
            d1.synchronize()
            ms[-1] += d0.elapsed_time(d1)
        return ms

    def arm_summary(mm, rr):
        return {"ms_per_step": statistics.mean(mm),
                "iters_per_step": statistics.mean(r["iters"] for r in rr),
                "learned_guess_used_fraction": sum(1 for r in rr if r["guess_used"] == 2) / len(rr)}

    # ---- our arm: learned guess + FP32/FP64 refinement
    sol = pkg.Solver(n, m=M, rtol=RTOL, precision="fp32_refine", guess="learned",
                     fallback="prev", warmup_steps=TAU0, seed=7 + rank,
                     grid_blocks=args.grid_blocks, **LEARN)
    tuning = sol.autotune(B[0])                          # launch shape (untimed, cached)
    warm = []
    run_series(sol, 0, TAU0, True, False, warm, drain=False)   # online warm-up (collect, train)
    run_series(sol, TAU0, W, True, False, warm, drain=False)   # benchmark warm-up
    res = []
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    barrier()
    l0 = pkg.kernel_launches()
    t_wall0 = time.perf_counter()
    ms = run_series(sol, TAU0 + W, K, True, True, res)
    train_host_ms = host_train[0] * 1e3
    barrier()
    t_wall = time.perf_counter() - t_wall0
    launches = pkg.kernel_launches() - l0
    clk = clocks.stop()
    value = aggregate_ms_per_step(sum(ms), K, world, dist, dev)
    # Algorithm 1's retention after tau0 (the paper: about 1 in 10 steps)
    post = warm[TAU0:] + res
    retained = {"admitted": sum(r["admitted"] for r in post), "steps": len(post)}

    # roofline of the dominant kernel (the persistent solver)
    hbm, peak_kind = peaks()
    byts = sum(algorithmic_bytes(r, N, M, 4) for r in res)
    byts2 = sum(two_pass_bytes(r, N, M, 4) for r in res)
    tos = sum(r["tos_ms"] for r in res)
    achieved = byts / (tos * 1e-3) / 1e9
    traffic = DRAM_BYTES_PER_STEP * statistics.mean(r["iters"] for r in res)
    us_step = 1e3 * tos / max(1, sum(r["iters"] for r in res))
    # the step's latency floor: its two group exchanges alone at the same CTA count
    # (None when the probe cannot run, e.g. its co-residency check under a profiler)
    try:
        floor_us = pkg.exchange_floor(tuning["grid_blocks"], M, 3000)
    except pkg.MLGMRESError as e:
        print("exchange floor probe unavailable: %s" % e, file=sys.stderr)
        floor_us = None

    # ---- end to end through the public API with host buffers
    Bh = torch.stack([torch.as_tensor(gen.rhs(t)) for t in range(TAU0 + W + K, TAU0 + W + 2 * K)])
    Bh = Bh.pin_memory()
    xh = torch.empty(N, dtype=torch.float64).pin_memory()
    bd = torch.empty(N, dtype=torch.float64, device=dev)
    xd = torch.empty(N, dtype=torch.float64, device=dev)
    barrier()
    t0 = time.perf_counter()
    for i in range(K):
        t = TAU0 + W + K + i
        bd.copy_(Bh[i], non_blocking=True)
        _, r = sol.solve(bd, xd)
        if (t + 1) % TRAIN_EVERY == 0:
            sol.train_step(stream=side)
        xh.copy_(xd, non_blocking=True)
        main.synchronize()
    side.synchronize()
    barrier()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, dist, dev)

    # ---- comparison arms on the same GPU and the same time steps
    compare = {}
    gains = {}
    if not args.no_compare:
        # the method against the same solver without the x_{t-1} fallback: the
        # network's guess competes with x0 = 0 only
        s3 = pkg.Solver(n, m=M, rtol=RTOL, precision="fp32_refine", guess="learned",
                        fallback="zero", warmup_steps=TAU0, **LEARN,
                        seed=11 + rank)
        s3.autotune(B[0])
        tmp = []
        run_series(s3, 0, TAU0 + W, True, False, tmp, drain=False)
        rr = []
        mm = run_series(s3, TAU0 + W, K, True, True, rr)
        compare["learned_fallback_zero"] = arm_summary(mm, rr)
        s3.close()
        for name, kw in (("plain_fp64_zero", dict(precision="fp64", guess="zero")),
                         ("plain_fp64_prev", dict(precision="fp64", guess="prev")),
                         ("fp32_refine_zero", dict(precision="fp32_refine", guess="zero")),
                         ("fp32_refine_prev", dict(precision="fp32_refine", guess="prev"))):
            s2 = pkg.Solver(n, m=M, rtol=RTOL, **kw)
            s2.autotune(B[0])
            tmp = []
            run_series(s2, TAU0 + W - 1, 1, False, False, tmp)  # primes PREV with x_{t-1}
            rr = []
            mm = run_series(s2, TAU0 + W, K, False, True, rr)
            compare[name] = arm_summary(mm, rr)
            s2.close()

        # control: the guess's 32 damped-Jacobi sweeps from x0 = 0, no network
        def smoothed_zero(solver, b):
            x = torch.zeros_like(b)
            return solver.smooth(b, x, SMOOTH)
        s4 = pkg.Solver(n, m=M, rtol=RTOL, precision="fp32_refine", guess="user",
                        guess_omega=0.8)
        s4.autotune(B[0])
        rr = []
        mm = run_series(s4, TAU0 + W, K, False, True, rr, pre=smoothed_zero)
        compare["smooth_only_zero"] = arm_summary(mm, rr)
        s4.close()
        lz = compare["learned_fallback_zero"]
        gains = {
            # > 1: the arm in the numerator is slower (the learned one wins)
            "learned_vs_fp32_refine_prev_ms_ratio":
                compare["fp32_refine_prev"]["ms_per_step"] / value,
            "learned_fallback_zero_vs_fp32_refine_zero_ms_ratio":
                compare["fp32_refine_zero"]["ms_per_step"] / lz["ms_per_step"],
            "learned_fallback_zero_vs_smooth_only_zero_ms_ratio":
                compare["smooth_only_zero"]["ms_per_step"] / lz["ms_per_step"],
            "learned_fallback_zero_vs_smooth_only_zero_iters_ratio":
                compare["smooth_only_zero"]["iters_per_step"] / lz["iters_per_step"],
            "learned_vs_plain_fp64_zero_ms_ratio":
                compare["plain_fp64_zero"]["ms_per_step"] / value,
        }

    # ---- the HBM-bound case: a capped 2048^2 FP32 solve at the autotuned shape
    roof_hbm = None
    if not args.no_hbm:
        from synthetic import RandomWalkSources2D
        gw = RandomWalkSources2D(HBM_N, 3001)
        bw = torch.as_tensor(gw.rhs(0)).to(dev)
        s5 = pkg.Solver(HBM_N, m=HBM_M, rtol=RTOL, precision="fp32_refine", guess="zero",
                        max_iters=HBM_STEPS)
        tw = s5.autotune(bw)
        rr = []
        for rep in range(2):            # the first run warms up; V (688 MB) exceeds L2
            flush.fill_(float(rep))
            _, r5 = s5.solve(bw)
            rr = [r5]
        NN = HBM_N * HBM_N
        b5 = algorithmic_bytes(rr[0], NN, HBM_M, 4)
        a5 = b5 / (rr[0]["tos_ms"] * 1e-3) / 1e9
        roof_hbm = {"bound": "hbm", "achieved": a5, "peak": hbm, "unit": "GB/s",
                    "frac": a5 / hbm, "peak_source": peak_kind,
                    "traffic": DRAM_BYTES_PER_STEP_2048 * rr[0]["iters"],
                    "frac_two_pass": two_pass_bytes(rr[0], NN, HBM_M, 4)
                    / (rr[0]["tos_ms"] * 1e-3) / 1e9 / hbm,
                    "workload": "2048x2048 random-walk sources (16 Gaussians + sin*sin mode, seed "
                                "3001), GMRES(40) FP32 cycles, one solve from x0 = 0 capped at "
                                "%d Arnoldi steps" % HBM_STEPS,
                    "arnoldi_steps": rr[0]["iters"], "kernel_ms": rr[0]["tos_ms"],
                    "us_per_arnoldi_step": 1e3 * rr[0]["tos_ms"] / max(rr[0]["iters"], 1),
                    "algorithmic_bytes": b5,
                    "launch_shape": {"ctas": tw["grid_blocks"], "v_stages": tw["v_stages"],
                                     "compact": tw["compact"]}}
        s5.close()

    # ---- the 3D variable-coefficient workload: a capped 192^3 solve
    roof_3d = None
    if not args.no_hbm:
        roof_3d = roofline_3d(pkg, torch, dev, hbm, peak_kind)

    # ---- single GPU: full time steps of the 2048^2 workload (error against DST)
    # and the 512-instance batched workload
    c3 = run_c3(pkg, torch, dev, args.c3_steps) if world == 1 and args.c3_steps > 0 else None
    c4 = run_c4(pkg, torch, dev) if world == 1 and not args.no_batch else None
    c5 = run_c5(pkg, torch, dev, args.c5_steps) if world == 1 and args.c5_steps > 0 else None

    line = None
    if rank == 0:
        used = sum(1 for r in res if r["guess_used"] == 2)
        line = {
            "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": value, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "guess": "learned network guess, kept only when its residual after one "
                                "GMRES(30) cycle beats the fallback x_{t-1}'s (it did on %d of "
                                "%d timed steps; the others ran from x_{t-1})" % (used, len(res)),
                       "precision": "fp32 Arnoldi cycles, fp64 restart residual / solution / "
                                    "Givens (iterative refinement)",
                       "network": "multi-scale conv net, 32 channels, bf16 operands, fp32 accum",
                       "online_warmup_steps": TAU0, "train_every": TRAIN_EVERY,
                       "train_phase": "64 Adam steps (lr 2e-3), minibatch 8, 64-pair replay ring, "
                                      "on a low-priority stream beside the solves",
                       "guess_smoothing": "%d damped-Jacobi sweeps (omega 0.8)" % SMOOTH,
                       "l2": "flushed between timed steps (256 MB write, outside the events)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "iters_per_step": statistics.mean(r["iters"] for r in res),
            "learned_guess_used_fraction": used / len(res),
            "relres_true_max": max(r["relres_true"] for r in res),
            "retained_after_tau0": dict(retained, fraction=retained["admitted"] / max(1, retained["steps"])),
            "compare": compare,
            "learned_gain": gains,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "frac_two_pass": byts2 / (tos * 1e-3) / 1e9 / hbm,
                         "algorithmic_bytes_per_step": byts / len(res),
                         "kernel": "gmres_persistent (FP32 variant, V in shared memory)",
                         "peak_source": peak_kind,
                         "note": "at 256^2 each CTA's slice of V sits in shared memory and the work "
                                 "vectors in L2: the algorithmic bytes are served on chip and the "
                                 "kernel is latency-bound; roofline_hbm is the HBM-bound case",
                         "launch_shape": {"ctas": tuning["grid_blocks"],
                                          "v_stages": tuning["v_stages"]},
                         "us_per_arnoldi_step": us_step,
                         "latency_floor_us": floor_us,
                         "floor_note": "latency_floor_us: the step's two group exchanges (CTA "
                                       "partials, group barrier, gather) alone, same CTA count, "
                                       "no passes"},
            "roofline_hbm": roof_hbm,
            "roofline_3d": roof_3d,
            "e2e": {"value": e2e_ms / (K * world), "unit": "ms",
                    "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N},
            "gpu_launches": launches,
            "clocks": clk,
            "wall_ms_per_step": t_wall * 1e3 / K,
            "train_step_host_ms_per_step": train_host_ms / K,
        }
        if c3 is not None:
            line["c3_full_steps"] = c3
        if c4 is not None:
            line["c4_batch"] = c4
        if c5 is not None:
            line["c5_full_steps"] = c5
        if world == 1 and not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(gen.rhs(TAU0 + W), n, TAU0 + W)
        else:
            line["cpu_baseline"] = None
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def roofline_3d(pkg, torch, dev, hbm, peak_kind, n=192, m=50, steps=300):
    """One 192^3 variable-kappa solve (log-normal kappa, seed 5001; the moving
    3D Gaussians at t = 0), GMRES(50) FP32 cycles from x0 = 0 capped at
    `steps` Arnoldi steps, at the autotuned shape; the second of two runs."""
    from synthetic import MovingGaussians3D, lognormal_kappa
    kap = lognormal_kappa(n, 5001).astype("float32")
    b = torch.as_tensor(MovingGaussians3D(n, 5001, 200).rhs(0)).to(dev)
    s = pkg.Solver(n, dim=3, kappa=kap, m=m, rtol=RTOL, precision="fp32_refine", guess="zero",
                   max_iters=steps)
    tw = s.autotune(b)
    r = None
    for _ in range(2):
        _, r = s.solve(b)
    s.close()
    N = n ** 3
    byts = algorithmic_bytes(r, N, m, 4, kappa=True)
    ach = byts / (r["tos_ms"] * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "peak_source": peak_kind, "traffic": DRAM_BYTES_PER_STEP_3D * r["iters"],
            # the bytes the two-pass step moves, with the four FP32 face
            # coefficient arrays in place of kappa
            "frac_two_pass": (two_pass_bytes(r, N, m, 4) + 16.0 * N * r["iters"])
            / (r["tos_ms"] * 1e-3) / 1e9 / hbm,
            "workload": "192^3 variable kappa (log-normal, seed 5001), 7-point, GMRES(50) FP32 "
                        "cycles, one solve from x0 = 0 capped at %d Arnoldi steps" % steps,
            "arnoldi_steps": r["iters"], "kernel_ms": r["tos_ms"],
            "us_per_arnoldi_step": 1e3 * r["tos_ms"] / max(r["iters"], 1),
            "launch_shape": {"ctas": tw["grid_blocks"], "v_stages": tw["v_stages"],
                             "compact": tw["compact"]}}


def run_c3(pkg, torch, dev, steps):
    """Full time steps of the 2048^2 workload (GMRES(40), FP32 cycles with FP64
    refinement to 1e-10): the first from x0 = 0, the rest from x_{t-1}; per
    step the device time, the iterations and the error against the DST-I
    solution (the oracle's direct solver)."""
    import numpy as np
    from oracle import direct
    from synthetic import RandomWalkSources2D
    gw = RandomWalkSources2D(HBM_N, 3001)
    s = pkg.Solver(HBM_N, m=HBM_M, rtol=RTOL, precision="fp32_refine", guess="prev",
                   max_iters=5 * 10 ** 6)
    s.autotune(torch.as_tensor(gw.rhs(0)).to(dev))
    out = []
    for t in range(steps):
        bh = gw.rhs(t)
        x, r = s.solve(torch.as_tensor(bh).to(dev))
        xr = direct.dst_solve_2d(HBM_N, bh)
        err = float(np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr))
        out.append({"t": t, "ms": r["tos_ms"], "iters": r["iters"], "relres_true": r["relres_true"],
                    "err_vs_dst": err, "guess": "zero" if t == 0 else "x_{t-1}"})
    s.close()
    mean = statistics.mean(o["ms"] for o in out)
    return {"workload": "2048x2048 random-walk sources (seed 3001), GMRES(40) FP32 cycles + "
                        "FP64 refinement, rtol 1e-10; the first step from x0 = 0, later ones "
                        "from x_{t-1}", "steps": out,
            "ms_per_step_mean": mean,
            "T12_ms": {"value": 12 * mean, "extrapolated": len(out) < 12,
                       "how": "12 x the mean of the timed steps" if len(out) < 12 else "timed"}}


def run_c5(pkg, torch, dev, steps, n=192, m=50):
    """Full time steps of the 192^3 variable-coefficient workload (log-normal
    kappa, seed 5001; moving 3D Gaussians), GMRES(50) FP32 cycles + FP64
    refinement to 1e-10: the first from x0 = 0, later ones from x_{t-1}; per
    step the device time, iterations and the true FP64 residual (the
    certificate: no direct solver covers variable kappa at this size)."""
    from synthetic import MovingGaussians3D, lognormal_kappa
    kap = lognormal_kappa(n, 5001).astype("float32")
    gen = MovingGaussians3D(n, 5001, 200)
    s = pkg.Solver(n, dim=3, kappa=kap, m=m, rtol=RTOL, precision="fp32_refine", guess="prev",
                   max_iters=3 * 10 ** 6)
    s.autotune(torch.as_tensor(gen.rhs(0)).to(dev))
    out = []
    for t in range(steps):
        _, r = s.solve(torch.as_tensor(gen.rhs(t)).to(dev))
        out.append({"t": t, "ms": r["tos_ms"], "iters": r["iters"], "relres_true": r["relres_true"],
                    "us_per_arnoldi_step": 1e3 * r["tos_ms"] / max(1, r["iters"]),
                    "guess": "zero" if t == 0 else "x_{t-1}"})
    s.close()
    return {"workload": "192^3 variable kappa (log-normal, seed 5001), 7-point, GMRES(50) FP32 "
                        "cycles + FP64 refinement, rtol 1e-10", "steps": out}


def run_c4(pkg, torch, dev):
    """The batched workload: 512 independent 2D Poisson instances, sides
    U{64..512} (seed 4001 + i), each with its own moving-Gaussian right-hand
    side at t = 0, GMRES(30) FP32 cycles + FP64 refinement to rtol 1e-8, all
    in one persistent launch; a sample of 8 instances against DST-I."""
    import numpy as np
    from oracle import direct
    from synthetic import batched_instances
    inst = batched_instances(512)
    ns = [n for n, _ in inst]
    bs = [torch.as_tensor(b).to(dev) for _, b in inst]
    s = pkg.Solver(max(ns), m=30, rtol=1e-8, precision="fp32_refine", batch_slots=4096,
                   max_iters=10 ** 7)
    xs, res = s.solve_batch(ns, bs)
    errs = []
    for i in range(0, 512, 64):
        xr = direct.dst_solve_2d(ns[i], inst[i][1])
        errs.append(float(np.linalg.norm(xs[i].cpu().numpy() - xr) / np.linalg.norm(xr)))
    s.close()
    return {"workload": "512 instances, sides U{64..512} (seed 4001+i), GMRES(30) FP32 + FP64 "
                        "refinement, rtol 1e-8, one persistent launch",
            "launch_ms": res[0]["tos_ms"], "unknowns": sum(n * n for n in ns),
            "arnoldi_steps": sum(r["iters"] for r in res),
            "relres_true_max": max(r["relres_true"] for r in res),
            "status": sorted(set(r["status"] for r in res)),
            "err_vs_dst_sample_max": max(errs), "err_sample": "instances 0, 64, ..., 448"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
