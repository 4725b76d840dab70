#!/usr/bin/env python3
"""Benchmark of the CN-FV tau-preconditioned solver on one GB300.

Metric: Crank-Nicolson steps per second on the n = 256 symmetric workload
(16.8 M unknowns, alpha = beta = gamma = 0.7, k+ = k- = 1, dt = 1/20,
manufactured exp(-t) source, true relative residual 1e-8), mixed precision
(split-BF16 tcgen05 inner PCG, FP64 refinement, extrapolated initial guess),
with the plain-FP64 GPU path on the same GPU reported beside it, and the
batched workload (64 uneven non-symmetric problems, 10 CN steps each, one
lock-step batched solve vs a loop of single-problem calls) as a sub-object.

One bench step = one CN step: the source cell averages at t_{m-1/2}, the RHS
(2 A_N - A) u^{m-1} + dt F, and the refined PCG solve.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload (the single-instance solve does not shard without a collective);
value = N * K / max-over-ranks time.  --impl reference times the CPU oracle
on the same workload (rank 0 only).
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import tfde_inputs as inp  # noqa: E402

METRIC = "CN steps/s at 3D N=256, mixed+warm-start vs plain FP64, 1e-8 rel residual"
UNIT = "CN steps/s"
WORKLOAD = "n256_sym_exp"
KERNEL_SOURCES = ["paper_2511_21198_gb300/csrc/tfde_tc_kernel.cuh"]


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=None, help="override the grid size (testing only)")
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--fft-mixed-steps", type=int, default=5,
                    help="chained steps of TFDE_MIXED on the FFT passes at n = 255 and 480 (0: skip)")
    ap.add_argument("--c2-steps", type=int, default=50,
                    help="CN steps of the n = 128 non-symmetric workload, mixed vs plain FP64 (0 skips it)")
    ap.add_argument("--no-c3-protocol", action="store_true",
                    help="skip the n = 256 run with one warm-up step and steps m = 2..20 (T = 1)")
    ap.add_argument("--no-parity", action="store_true",
                    help="skip the full-size tight-residual comparison of the mixed and FP64 GPU paths")
    ap.add_argument("--no-spectra", action="store_true", help="skip the Lanczos spectra of the preconditioned systems")
    ap.add_argument("--no-comparisons", action="store_true",
                    help="skip the host-loop and grid-basis comparison problems (one problem on the device)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="budget of the oracle CPU baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch-count", type=int, default=64,
                    help="problems of the uneven batched workload (0 skips it)")
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--batch-guess-order", type=int, default=3,
                    help="initial guess of the batched workload's chained steps (as --guess-order)")
    ap.add_argument("--cnn-steps", type=int, default=100,
                    help="CN steps of the warm-start evaluation at n = 128 (0 skips training and evaluation)")
    ap.add_argument("--cnn-train-steps", type=int, default=2000, help="Adam steps of the warm-start training")
    ap.add_argument("--guess-order", type=int, default=3,
                    help="initial guess of the mixed path: 0 previous step, 1/2 polynomial extrapolation, "
                         "3 order 2 with its minimal-residual correction over the stored history")
    return ap.parse_args(argv)


# ----------------------------------------------------------------- distributed
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    if world <= 1:
        return False
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend=backend, init_method="env://")
    return True


def barrier(on):
    if on:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x: float, on: bool, device=None) -> float:
    """Maximum of a host scalar over all ranks (identity without a process group)."""
    if not on:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(steps_per_rank: int, world: int, max_seconds: float) -> float:
    """Whole-job throughput: all ranks' steps over the slowest rank's time."""
    return steps_per_rank * world / max_seconds


# ---------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------- helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs"), "bf16_tflops": d.get("bf16_tflops"),
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def workload_config(n: int, W: dict, dt: float, tol: float) -> dict:
    """The keys that name the workload, shared by both arms' JSON lines."""
    return {"workload": WORKLOAD, "n": n, "unknowns": n ** 3, "delta": list(W["delta"]),
            "k_plus": list(W["kp"]), "k_minus": list(W["km"]), "dt": dt, "tol": tol}


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per launch of the tcgen05 kernel from the committed ncu
    summary, or None when absent or taken on a different kernel source."""
    p = os.path.join(ROOT, "profiles", "axis_gemm_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_sha") != kernel_hash():
        return None
    return d.get("dram_bytes_per_launch_n256")


def survey_bytes_per_iteration(n: int) -> float:
    """Algorithmic bytes of the split contraction per inner Krylov iteration:
    the Toeplitz matvec reads p and writes A p, the preconditioner reads r
    and writes z, FP32 vectors of n^3 elements."""
    return 4.0 * n ** 3 * 4


def survey_bytes_per_step(n: int, iters: float, sweeps: float) -> float:
    """Algorithmic bytes of one CN step: 13 FP32 vector passes per inner
    iteration (matvec 2, x/r update 6, preconditioner 2, direction 3), the
    right-hand side (3 FP64 passes) and one FP64 residual per refinement
    sweep (4 FP64 passes)."""
    N = float(n) ** 3
    return iters * 13 * N * 4 + 3 * N * 8 + sweeps * 4 * N * 8


def source_factors(t: float):
    """Time factors (cP, cS) = (phi'(t), -phi(t)) of the exp(-t) manufactured source."""
    e = math.exp(-t)
    return -e, -e


# ---------------------------------------------------------------- CPU oracle
def oracle_steps(n, delta, k, dt, tol, budget_s, max_steps=None, with_iters=False):
    """Run oracle CN steps from the manufactured initial data until the time
    budget is used (at least one step); returns (steps, seconds), and with
    with_iters=True (steps, seconds, PCG iterations)."""
    from oracle import tfde_oracle as o
    prob = o.Problem(n=(n, n, n), delta=delta, kp=k, km=k, dt=dt)
    tau = o.build_tau(prob)
    u = inp.example2_initial(n)
    steps, iters, t0 = 0, 0, time.perf_counter()
    while True:
        th = (steps + 0.5) * dt
        F = o.source_cell_average(prob, th, "exp")
        b = o.rhs(prob, u, F)
        u, info = o.pcg(lambda v: o.apply_A(prob, v), lambda r: o.apply_Pinv(tau, r), b, u, tol, 10 ** 6)
        steps += 1
        iters += info.iters
        el = time.perf_counter() - t0
        if el >= budget_s or (max_steps and steps >= max_steps):
            return (steps, el, iters) if with_iters else (steps, el)


def oracle_iteration_seconds(n, delta, k, dt):
    """Seconds of one oracle PCG iteration's operator and preconditioner
    application, and of one right-hand side, on the n^3 workload (numpy FP64,
    as many BLAS threads as the process is given)."""
    from oracle import tfde_oracle as o
    prob = o.Problem(n=(n, n, n), delta=delta, kp=k, km=k, dt=dt)
    tau = o.build_tau(prob)
    u = inp.example2_initial(n)
    t0 = time.perf_counter()
    o.rhs(prob, u, None)
    t1 = time.perf_counter()
    v = o.apply_A(prob, u)
    o.apply_Pinv(tau, v)
    t2 = time.perf_counter()
    return t2 - t1, t1 - t0


def oracle_one_core(n, delta, k, dt, iters_per_step):
    """The oracle's CN steps/s on one host core: one iteration's operator and
    preconditioner and one right-hand side timed in a child process pinned
    to one core with one BLAS thread, scaled by the iterations per step."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[v] = "1"
    code = ("import json, os, sys; sys.path.insert(0, %r); os.sched_setaffinity(0, {min(os.sched_getaffinity(0))}); "
            "import bench; print(json.dumps(bench.oracle_iteration_seconds(%d, %r, %r, %r)))"
            % (ROOT, n, tuple(delta), tuple(k), dt))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return None
    it_s, rhs_s = json.loads(r.stdout.strip().splitlines()[-1])
    step_s = rhs_s + iters_per_step * it_s
    return {"value": 1.0 / step_s, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one operator + preconditioner application ({it_s:.1f} s) and one right-hand side "
                      f"({rhs_s:.1f} s) of the n={n} workload on one core with one BLAS thread, scaled by "
                      f"{iters_per_step:.1f} PCG iterations per step (the all-core sample's count)"}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


# ----------------------------------------------------------------- our arm
def chained_steps(T, h, u, F, dt, m0, count, tol, stream):
    """`count` chained in-place CN steps m0+1 .. m0+count of the exp(-t)
    manufactured workload (source assembled on the device each step); the
    chain restarts when m0 == 0.  Returns (inner iterations, refinement
    sweeps, largest final relative residual)."""
    iters = sweeps = 0
    relres = 0.0
    for i in range(count):
        cP, cS = source_factors((m0 + i + 0.5) * dt)
        T.tfde_source_example2(h, cP, cS, F, stream)
        info = T.tfde_cn_advance(h, u, F, m0 + i == 0, tol, stream)
        iters += info.iters
        sweeps += info.refine_sweeps
        relres = max(relres, info.relres)
    return iters, sweeps, relres


def run_ours(args):
    import torch

    from paper_2511_21198_gb300 import tfde as T

    world, rank, local = dist_env()
    on = dist_init(world, "nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    T.load()
    W = inp.WORKLOADS[WORKLOAD]
    n = args.n or W["n"]
    M = W["M"]
    dt = 1.0 / M
    tol = W["tol"]
    params = T.make_params((n, n, n), W["delta"], W["kp"], W["km"], dt)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    u0 = torch.from_numpy(inp.example2_initial(n)).to(dev)
    # ---- mixed precision (the metric)
    h = T.tfde_assemble(params, T.TFDE_MIXED, stream)
    T.tfde_set_guess_order(h, args.guess_order)
    u, F = u0.clone(), torch.empty_like(u0)
    chained_steps(T, h, u, F, dt, 0, args.warmup, tol, stream)
    torch.cuda.synchronize()
    barrier(on)
    # the product path as is: no per-launch timing events (those would also
    # switch the inner PCG to its host-driven loop)
    T.tfde_stats_reset(time_tc=False)
    clk = ClockSampler(local)
    clk.start()
    torch.cuda.synchronize()
    e0.record(stream)
    iters, sweeps, relres = chained_steps(T, h, u, F, dt, args.warmup, args.steps, tol, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    barrier(on)
    ms = e0.elapsed_time(e1)
    launches = int(T.tfde_stats_get().kernel_launches)
    ms_max = reduce_max(ms, on, dev)
    value = aggregate_value(args.steps, world, ms_max / 1e3)
    t_end = (args.warmup + args.steps) * dt
    exact = torch.from_numpy(inp.example2_initial(n, math.exp(-t_end))).to(dev)
    err = float((u - exact).abs().max() / exact.abs().max())
    u_end = u.clone()

    # ---- end to end through the C ABI with host buffers (copies timed)
    e2e = None
    if not args.no_e2e:
        host_u = u.cpu().pin_memory()
        host_out = torch.empty_like(host_u).pin_memory()
        m0 = args.warmup + args.steps
        torch.cuda.synchronize()
        barrier(on)
        e0.record(stream)
        for i in range(args.steps):
            # u^{m-1} from the host buffer, u^m back to the other one, through the
            # library's host-buffer step (its copies overlap the step's own work;
            # the host copy holds exactly the previous output, so the chain stays valid)
            cP, cS = source_factors((m0 + i + 0.5) * dt)
            T.tfde_source_example2(h, cP, cS, F, stream)
            T.tfde_cn_advance_host(h, host_u, host_out, u, F, False, tol, stream)
            host_u, host_out = host_out, host_u
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(on)
        ms_e = reduce_max(e0.elapsed_time(e1), on, dev)
        nbytes = u.numel() * u.element_size()
        e2e = {"value": aggregate_value(args.steps, world, ms_e / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}

    # ---- kernel timing for the roofline: the same chained steps with every
    # tensor-core launch bracketed by CUDA events (host-driven inner loop)
    m0 = args.warmup + 2 * args.steps
    T.tfde_stats_reset(time_tc=True)
    e0.record(stream)
    it_t, sw_t, _ = chained_steps(T, h, u, F, dt, m0, args.steps, tol, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_t = e0.elapsed_time(e1)
    st = T.tfde_stats_get()
    T.tfde_stats_reset(time_tc=False)
    host_gap = inner_basis = None
    if not args.no_comparisons:
        # ---- host gap: a second problem marches the same trajectory (warm-up and
        # timed steps) with the inner loop driven from the host; the iterates are
        # the same, so the time difference is the host round trips
        hb = T.tfde_assemble(params, T.TFDE_MIXED, stream)
        T.tfde_set_guess_order(hb, args.guess_order)
        T.tfde_set_device_loop(hb, False)
        ub = u0.clone()
        chained_steps(T, hb, ub, F, dt, 0, args.warmup, tol, stream)
        torch.cuda.synchronize()
        e0.record(stream)
        it_h, _, _ = chained_steps(T, hb, ub, F, dt, args.warmup, args.steps, tol, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_h = e0.elapsed_time(e1)
        T.tfde_destroy(hb)
        del ub
        # ---- the same steps with the inner PCG in the grid basis (tfde_set_spectral_inner(h, 0))
        hg = T.tfde_assemble(params, T.TFDE_MIXED, stream)
        T.tfde_set_guess_order(hg, args.guess_order)
        T.tfde_set_spectral_inner(hg, False)
        ug = u0.clone()
        chained_steps(T, hg, ug, F, dt, 0, args.warmup, tol, stream)
        torch.cuda.synchronize()
        e0.record(stream)
        it_g, _, rr_g = chained_steps(T, hg, ug, F, dt, args.warmup, args.steps, tol, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_g = e0.elapsed_time(e1)
        T.tfde_destroy(hg)
        del ug
        inner_basis = {"ms_per_step_eigenbasis": ms / args.steps, "ms_per_step_grid_basis": ms_g / args.steps,
                       "iters_per_step_eigenbasis": iters / args.steps, "iters_per_step_grid_basis": it_g / args.steps,
                       "max_relres_grid_basis": rr_g,
                       "note": "the timed steps again on a problem whose inner PCG iterates in the grid basis "
                               "(operator 3 and preconditioner 6 split launches per iteration) instead of the "
                               "sine-transform eigenbasis (3 split launches per iteration)"}
        host_gap = {"ms_per_step_device_loop": ms / args.steps, "ms_per_step_host_loop": ms_h / args.steps,
                    "iters_per_step_host_loop": it_h / args.steps, "iters_per_step_device_loop": iters / args.steps,
                    "host_gap_share_removed": (ms_h - ms) / ms_h,
                    "note": "the timed steps again on a second problem with the inner PCG driven from the host "
                            "(one blocking read of <r, r> per inner iteration) instead of one graph launch per "
                            "refinement sweep"}
    # ---- the survey's C-3 protocol: one warm-up step, then steps m = 2 .. 20
    # (T = 1), CN steps/s from the median of 5 runs from u0
    c3 = None
    if not args.no_c3_protocol and args.n is None:
        runs = []
        for rep in range(5):
            u = u0.clone()
            chained_steps(T, h, u, F, dt, 0, 1, tol, stream)
            torch.cuda.synchronize()
            e0.record(stream)
            it3, sw3, rr3 = chained_steps(T, h, u, F, dt, 1, M - 1, tol, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            runs.append((e0.elapsed_time(e1), it3, sw3, rr3))
        runs.sort(key=lambda t: t[0])
        ms3, it3, sw3, rr3 = runs[len(runs) // 2]
        ex3 = torch.from_numpy(inp.example2_initial(n, math.exp(-1.0))).to(dev)
        c3 = {"value": (M - 1) / (ms3 / 1e3), "unit": UNIT, "warmup_steps": 1, "timed_steps": f"m = 2..{M}",
              "runs": len(runs), "statistic": "median of the runs",
              "ms_per_step_runs": [r[0] / (M - 1) for r in runs],
              "ms_per_step": ms3 / (M - 1), "iters_per_step": it3 / (M - 1),
              "refine_sweeps_per_step": sw3 / (M - 1), "max_relres": max(r[3] for r in runs),
              "max_rel_err_vs_exact_at_T1": float((u - ex3).abs().max() / ex3.abs().max())}
    T.tfde_destroy(h)

    # ---- plain FP64 path on the same GPU (comparison)
    fp64 = None
    if args.fp64_steps > 0:
        h64 = T.tfde_assemble(params, T.TFDE_FP64, stream)
        T.tfde_set_guess_order(h64, args.guess_order)
        u = u0.clone()
        chained_steps(T, h64, u, F, dt, 0, 1, tol, stream)
        torch.cuda.synchronize()
        e0.record(stream)
        it64, _, rr64 = chained_steps(T, h64, u, F, dt, 1, args.fp64_steps, tol, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = reduce_max(e0.elapsed_time(e1), on, dev)
        fp64 = {"value": aggregate_value(args.fp64_steps, world, ms64 / 1e3), "unit": UNIT,
                "ms_per_step": ms64 / args.fp64_steps, "iters_per_step": it64 / args.fp64_steps,
                "steps": args.fp64_steps, "warmup_steps": 1, "max_relres": rr64,
                "initial_guess": "as the mixed path"}
        T.tfde_destroy(h64)

    # ---- full-size parity: mixed and FP64 GPU paths from the same state, tight residual
    parity = None
    if not args.no_parity:
        parity = full_size_parity(T, params, u_end, (args.warmup + args.steps + 0.5) * dt, dev, stream)

    # ---- TFDE_MIXED on the FFT passes (grids the tensor-core path does not take)
    fftm = None
    if args.fft_mixed_steps > 0 and args.n is None:
        fftm = run_fft_mixed(T, args.fft_mixed_steps, args.guess_order, dev, stream)

    # ---- the non-symmetric workload: n = 128, PGMRES(20), mixed vs plain FP64
    c2 = None
    if args.c2_steps > 0 and args.n is None:
        c2 = run_c2(T, args.c2_steps, args.guess_order, dev, stream, check_oracle=rank == 0)

    # ---- spectra of the preconditioned systems at the benchmark sizes (Sec. 3)
    spectra = None
    if not args.no_spectra and args.n is None:
        spectra = run_spectra(T, dev, stream)

    # ---- batched workload: uneven problems, lock-step batched solve vs a loop
    batched = None
    if args.batch_count > 0 and args.batch_steps > 0:
        batched = run_batched(T, args.batch_count, args.batch_steps, dev, stream, args.batch_guess_order)

    # ---- learned warm start: train at n = 64, evaluate at n = 128
    warm = None
    if args.cnn_steps > 0 and args.cnn_train_steps > 0:
        warm = run_warm_start(T, args.cnn_train_steps, args.cnn_steps, dev, stream)

    # ---- roofline of the dominant kernel (tcgen05 per-axis contraction)
    peaks = measured_peaks()
    roof = None
    ks = st.kind[T.TFDE_KIND_SPLIT]
    kx = st.kind[T.TFDE_KIND_EXACT]
    if ks.timed > 0 and ks.ms > 0:
        # dominant kernel: the split-BF16 per-axis contraction (fast operator and
        # preconditioner of every inner iteration), timed alone by event pairs.
        # frac: the algorithmic bytes of the inner iterations (matvec read p,
        # write Ap; preconditioner read r, write z; FP32) over the summed
        # launch time; schedule_frac: the bytes the launches' schedule moves.
        alg = it_t * survey_bytes_per_iteration(n)
        achieved = alg / (ks.ms / 1e3) / 1e9
        sched = ks.bytes / (ks.ms / 1e3) / 1e9
        step_bytes = survey_bytes_per_step(n, iters / args.steps, sweeps / args.steps)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": recorded_traffic(),
                "kernel": "tfde::tc::axis_gemm_kernel", "peak_source": peaks["source"] + " (hbm_gbs)",
                "launches": int(ks.launches), "avg_launch_us": 1e3 * ks.ms / ks.timed,
                "algorithmic_bytes_per_launch": alg / ks.launches,
                "algorithmic_bytes_basis": "16 n^3 bytes per inner iteration (FP32 matvec p -> Ap, "
                                           "preconditioner r -> z)",
                "split_us_per_inner_iteration": 1e3 * ks.ms / max(it_t, 1),
                "timing_run": f"{args.steps} further chained steps with CUDA-event pairs around every "
                              f"tensor-core launch ({ms_t / args.steps:.3f} ms/step, {it_t / args.steps:.2f} "
                              "inner iterations per step)",
                "schedule_bytes_per_launch": ks.bytes / ks.launches, "schedule_achieved": sched,
                "schedule_frac": sched / peaks["hbm_gbs"],
                "tensor_tflops": ks.flops / (ks.ms / 1e3) / 1e12,
                "kernel_share_of_step": ks.ms / ms_t,
                "step": {"algorithmic_bytes_per_step": step_bytes,
                         "achieved": step_bytes / (ms / args.steps / 1e3) / 1e9,
                         "frac": step_bytes / (ms / args.steps / 1e3) / 1e9 / peaks["hbm_gbs"]}}
        if kx.timed > 0 and kx.ms > 0:
            roof["exact_residual_kernel"] = {
                "kernel": "tfde::oz::oz_gemm_kernel", "bound": "tensor", "launches": int(kx.launches),
                "avg_launch_us": 1e3 * kx.ms / kx.timed,
                "tensor_tflops": kx.flops / (kx.ms / 1e3) / 1e12,
                "frac_of_bf16_peak": kx.flops / (kx.ms / 1e3) / 1e12 / peaks["bf16_tflops_sustained"],
                "achieved_gbs": kx.bytes / (kx.ms / 1e3) / 1e9,
                "kernel_share_of_step": kx.ms / ms_t}

    # ---- CPU baseline (oracle), rank 0 at N = 1 only
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        steps_c, sec, it_c = oracle_steps(n, W["delta"], W["kp"], dt, tol, args.cpu_seconds, with_iters=True)
        cpu = {"value": steps_c / sec, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": f"{steps_c} CN step(s) of the n={n} workload by the numpy FP64 oracle "
                         f"(PCG, x0 = u^(m-1), {it_c / steps_c:.1f} iterations per step), {sec:.1f} s"}
        one = oracle_one_core(n, W["delta"], W["kp"], dt, it_c / steps_c)
        if one:
            cpu["one_core"] = one

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16-split/fp32 inner, fp64 refinement",
            "data": "synthetic: manufactured solution exp(-t) x^2(1-x)^2 y^2(1-y)^2 z^2(1-z)^2",
            "config": {**workload_config(n, W, dt, tol),
                       "solver": "PCG(tau) inner FP32 / split-BF16 tcgen05, FP64 iterative refinement",
                       "warm_start": ("none: previous step u^(m-1)" if args.guess_order == 0 else
                                      "extrapolated (not learned): "
                                      f"order-{min(args.guess_order, 2)} polynomial extrapolation in time"
                                      + (" with a minimal-residual correction over the history differences"
                                         if args.guess_order >= 3 else "")
                                      + " (A x0 from stored A u, no extra operator application); the learned "
                                        "network's comparison is the warm_start sub-object"),
                       "step_api": "tfde_cn_advance (chained: A u^(m-1) = b^(m-1) - r^(m-1))",
                       "l2": "inputs larger than L2 (each FP64 vector 134 MB, working set > 2 GB)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "host_gap": host_gap, "inner_basis": inner_basis,
            "clocks": clocks, "fp64_path": fp64, "c3_protocol": c3, "parity_n256": parity,
            "c2_nonsymmetric_n128": c2, "mixed_fft_path": fftm, "batched": batched, "warm_start": warm, "spectra": spectra,
            "iters_per_step": iters / args.steps, "refine_sweeps_per_step": sweeps / args.steps,
            "max_relres": relres, "max_rel_err_vs_exact": err,
        }
        print(json.dumps(line), flush=True)
    if on:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_spectra(T, dev, stream, steps=40):
    """Lanczos estimates (tfde_spectrum, FP64) of the preconditioned
    systems' spectra on the n = 256 symmetric and n = 128 non-symmetric
    workloads, beside the paper's grid-independent bounds."""
    import torch
    out = {"lanczos_steps": steps}
    for key in ("n256_sym_exp", "n128_nonsym"):
        W = inp.WORKLOADS[key]
        n = W["n"]
        v0 = torch.from_numpy(inp.uniform_vector((n, n, n), 10)).to(dev)
        t0 = time.perf_counter()
        s = T.tfde_spectrum(T.make_params((n, n, n), W["delta"], W["kp"], W["km"], 1.0 / W["M"]), steps, v0, stream)
        out[key] = {"sym_min": s.sym_min, "sym_max": s.sym_max, "paper_sym_interval": [0.5, 1.5],
                    "skew_rho": s.skew_rho, "paper_varsigma": s.varsigma, "paper_omega": s.omega,
                    "omega_from_estimates": s.omega_est, "seconds": time.perf_counter() - t0}
        del v0
    return out


def full_size_parity(T, params, u_prev, t_half, dev, stream):
    """One CN step from the same state u^{m-1} through the mixed and the FP64
    GPU paths at a 1e-12 true residual (tfde_cn_step, x0 = u^{m-1}), and the
    mixed step at the benchmark's 1e-8: their relative 2-norm differences."""
    import torch
    out = {"state": "u^(m-1) after the timed steps", "tight_tol": 1e-12}
    hm = T.tfde_assemble(params, T.TFDE_MIXED, stream)
    h64 = T.tfde_assemble(params, T.TFDE_FP64, stream)
    try:
        F = torch.empty_like(u_prev)
        cP, cS = source_factors(t_half)
        T.tfde_source_example2(hm, cP, cS, F, stream)
        xm, x64, x8 = torch.empty_like(u_prev), torch.empty_like(u_prev), torch.empty_like(u_prev)
        im = T.tfde_cn_step(hm, u_prev, F, None, xm, 1e-12, stream)
        i64 = T.tfde_cn_step(h64, u_prev, F, None, x64, 1e-12, stream)
        i8 = T.tfde_cn_step(hm, u_prev, F, None, x8, 1e-8, stream)
        nrm = float(torch.linalg.vector_norm(x64))
        out.update({"rel_err_mixed_vs_fp64": float(torch.linalg.vector_norm(xm - x64)) / nrm,
                    "relres_mixed": im.relres, "relres_fp64": i64.relres,
                    "rel_err_tol1e8_vs_tight": float(torch.linalg.vector_norm(x8 - x64)) / nrm,
                    "relres_tol1e8": i8.relres})
    finally:
        T.tfde_destroy(hm)
        T.tfde_destroy(h64)
    return out


def run_fft_mixed(T, steps, guess_order, dev, stream, sizes=(255, 480)):
    """TFDE_MIXED on grids the tensor-core contraction does not take: FP32
    inner PCG on the FFT passes inside FP64 refinement (residual on the FP64
    FFT passes).  The symmetric manufactured workload's coefficients
    (delta = 0.7, k+- = 1, dt = 1/20, tol 1e-8) at n = 255 (not a multiple of
    8, next to the n = 256 headline) and n = 480 (above 448): `steps` chained
    CN steps after one warm-up step, against the plain FP64 path (FFT passes
    too) over 2 steps from the same state."""
    import torch
    W = inp.WORKLOADS[WORKLOAD]
    dt, tol = 1.0 / W["M"], W["tol"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for n in sizes:
        prm = T.make_params((n, n, n), W["delta"], W["kp"], W["km"], dt)
        u0 = torch.from_numpy(inp.example2_initial(n)).to(dev)
        F = torch.empty_like(u0)
        res = {"workload": f"n={n} symmetric, PCG, tol {tol:g}, {steps} chained steps after 1 warm-up",
               "unknowns": n ** 3}
        for name, prec, k in (("mixed_fft", T.TFDE_MIXED, steps), ("fp64_fft", T.TFDE_FP64, 2)):
            h = T.tfde_assemble(prm, prec, stream)
            try:
                T.tfde_set_guess_order(h, guess_order)
                u = u0.clone()
                chained_steps(T, h, u, F, dt, 0, 1, tol, stream)
                torch.cuda.synchronize()
                e0.record(stream)
                it, sw, rr = chained_steps(T, h, u, F, dt, 1, k, tol, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                res[name] = {"value": k / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / k, "steps": k,
                             "iters_per_step": it / k, "refine_sweeps_per_step": sw / k, "max_relres": rr}
            finally:
                T.tfde_destroy(h)
        res["speedup_mixed_vs_fp64"] = res["mixed_fft"]["value"] / res["fp64_fft"]["value"]
        out[f"n{n}"] = res
        del u0, F
        torch.cuda.empty_cache()
    return out


def run_c2(T, steps, guess_order, dev, stream, check_oracle=True):
    """The non-symmetric workload (n = 128, delta = (0.3, 0.6, 0.8), k+ = 1,
    k- = 0.5, f = 0, smoothed-noise u0 with seed 2, dt = 1/50, PGMRES(20),
    tol 1e-8): `steps` chained CN steps through the mixed path and through
    the plain FP64 path, each timed with CUDA events after one warm-up step,
    and their trajectories compared; the last mixed step is also compared
    with the oracle's GMRES step at a tight residual from the same state."""
    import torch
    Wc = inp.WORKLOADS["n128_nonsym"]
    n, dt, tol = Wc["n"], 1.0 / Wc["M"], Wc["tol"]
    prm = T.make_params((n, n, n), Wc["delta"], Wc["kp"], Wc["km"], dt)
    u0 = torch.from_numpy(inp.smoothed_uniform((n, n, n), Wc["u0_seed"])).to(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": "n=128 non-symmetric, PGMRES(20), f = 0, tol 1e-8", "steps": steps, "warmup_steps": 1}
    finals = {}
    prev_state = None
    for name, prec in (("mixed", T.TFDE_MIXED), ("fp64", T.TFDE_FP64)):
        h = T.tfde_assemble(prm, prec, stream)
        try:
            T.tfde_set_guess_order(h, guess_order)
            u = u0.clone()
            T.tfde_cn_advance(h, u, None, True, tol, stream)
            torch.cuda.synchronize()
            its, rr = 0, 0.0
            e0.record(stream)
            for m in range(1, steps):
                if name == "mixed" and m == steps - 1:
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms_part = e0.elapsed_time(e1)
                    prev_state = u.clone()
                    e0.record(stream)
                info = T.tfde_cn_advance(h, u, None, False, tol, stream)
                its += info.iters
                rr = max(rr, info.relres)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) + (ms_part if name == "mixed" else 0.0)
            finals[name] = u
            out[name] = {"value": (steps - 1) / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / (steps - 1),
                         "iters_per_step": its / (steps - 1), "max_relres": rr}
        finally:
            T.tfde_destroy(h)
    out["speedup_mixed_vs_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    out["rel_err_mixed_vs_fp64_trajectory"] = float(torch.linalg.vector_norm(finals["mixed"] - finals["fp64"])
                                                    / torch.linalg.vector_norm(finals["fp64"]))
    if check_oracle and prev_state is not None:
        from oracle import tfde_oracle as o
        op = o.Problem(n=(n, n, n), delta=Wc["delta"], kp=Wc["kp"], km=Wc["km"], dt=dt)
        up = prev_state.cpu().numpy()
        b = o.rhs(op, up, None)
        tau = o.build_tau(op)
        t0 = time.perf_counter()
        xo, _ = o.gmres_left(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, up, 1e-13, 4000,
                             restart=20, criterion="true")
        h = T.tfde_assemble(prm, T.TFDE_MIXED, stream)
        try:
            xm = torch.empty_like(prev_state)
            info = T.tfde_cn_step(h, prev_state, None, None, xm, 1e-12, stream)
            out["last_step_vs_oracle"] = {
                "rel_err_tight": float(np.linalg.norm(xm.cpu().numpy() - xo) / np.linalg.norm(xo)),
                "rel_err_tol1e8": float(np.linalg.norm(finals["mixed"].cpu().numpy() - xo) / np.linalg.norm(xo)),
                "relres_mixed_tight": info.relres, "oracle_tol": 1e-13, "oracle_s": time.perf_counter() - t0}
        finally:
            T.tfde_destroy(h)
    return out


def run_warm_start(T, train_steps, eval_steps, dev, stream):
    """The learned warm start: trajectories of the solver at n = 64 (128
    seeds, 8 steps each, random delta, k+-, dt in {0.005, 0.01, 0.02, 0.04},
    manufactured source), Adam on mini-batches of 8 samples with the two
    previous levels as history (the network corrects the order-2
    extrapolation in time), then `eval_steps` chained CN steps at n = 128
    (delta = (0.3, 0.6, 0.8), k+ = 1, k- = 0.5, dt = 0.01, f = 0,
    smoothed-noise u0, tol 1e-8) with the network's guess (started from the
    least-residual point between u^m and it) against the previous-step guess
    and the order-3 corrected extrapolation.  Timed with CUDA events."""
    import torch

    from paper_2511_21198_gb300 import warmstart as W
    t0 = time.time()
    ntraj, nsteps = 128, 8
    data = W.generate_trajectories(64, list(range(100, 100 + ntraj)), nsteps, [0.005, 0.01, 0.02, 0.04],
                                   with_source=True, stream=stream, device=dev)
    net = T.tfde_cnn_create((64, 64, 64))
    try:
        T.tfde_cnn_set_params(net, W.init_params(0))
        torch.cuda.synchronize()
        t1 = time.time()
        hist = W.train(net, data, train_steps, 8, 2e-3, 0, stream)
        torch.cuda.synchronize()
        t2 = time.time()
        params = T.tfde_cnn_get_params(net)
    finally:
        T.tfde_cnn_destroy(net)
    del data
    n, dt = 128, 0.01
    d, kp, km = (0.3, 0.6, 0.8), (1.0,) * 3, (0.5,) * 3
    prm = T.make_params((n, n, n), d, kp, km, dt)
    coef = W.coefficients(prm)
    u0 = torch.from_numpy(inp.smoothed_uniform((n, n, n), 5)).to(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"train": {"grid": 64, "trajectories": ntraj, "samples": ntraj * (nsteps - 2), "history_levels": 2,
                     "adam_steps": train_steps, "batch": 8,
                     "loss_first10": float(np.mean(hist[:10])), "loss_last10": float(np.mean(hist[-10:])),
                     "data_s": t1 - t0, "train_s": t2 - t1},
           "eval": {"grid": n, "steps": eval_steps, "tol": 1e-8}}
    ne = T.tfde_cnn_create((n, n, n))
    T.tfde_cnn_set_params(ne, params)
    try:
        for mode in ("previous_step", "extrapolated_order3", "network"):
            h = T.tfde_assemble(prm, T.TFDE_MIXED, stream)
            try:
                if mode == "extrapolated_order3":
                    T.tfde_set_guess_order(h, 3)
                u = u0.clone()
                x0 = torch.empty_like(u)
                hist = [u0.clone()]                                    # u^{m-1}, u^{m-2} for the network
                T.tfde_cn_advance(h, u, None, True, 1e-8, stream)     # step 1 (no guess yet)
                its, used, r0 = 0, 0, []
                torch.cuda.synchronize()
                e0.record(stream)
                for m in range(eval_steps):
                    if mode == "network":
                        u1 = hist[-1]
                        u2 = hist[-2] if len(hist) > 1 else None
                        T.tfde_cnn_predict_hist(ne, u, u1, u2, None, coef, x0, stream)
                        prev = u.clone()
                        info, ug = T.tfde_cn_advance_guess(h, u, None, x0, False, 1e-8, stream)
                        hist = [hist[-1], prev]
                        used += int(ug)
                    else:
                        info = T.tfde_cn_advance(h, u, None, False, 1e-8, stream)
                    its += info.iters
                    r0.append(info.relres0)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                out["eval"][mode] = {"iters_per_step": its / eval_steps, "ms_per_step": ms / eval_steps,
                                     "median_initial_relres": float(np.median(r0))}
                if mode == "network":
                    out["eval"][mode]["guess_used_steps"] = used
                    out["eval"][mode]["fallback_steps"] = eval_steps - used
            finally:
                T.tfde_destroy(h)
    finally:
        T.tfde_cnn_destroy(ne)
    ev = out["eval"]
    ev["network_vs_previous_step"] = {
        "iters_ratio": ev["network"]["iters_per_step"] / ev["previous_step"]["iters_per_step"],
        "ms_ratio": ev["network"]["ms_per_step"] / ev["previous_step"]["ms_per_step"]}
    ev["network_vs_extrapolated_order3"] = {
        "iters_ratio": ev["network"]["iters_per_step"] / ev["extrapolated_order3"]["iters_per_step"],
        "ms_ratio": ev["network"]["ms_per_step"] / ev["extrapolated_order3"]["ms_per_step"]}
    return out


def run_batched(T, count, steps, dev, stream, guess_order=0):
    """The uneven batched workload: `count` problems (n per axis from
    {32, 48, 64, 96, 128}, delta ~ U(0.1, 0.9), k+- ~ U(0.5, 2), seed 4),
    smoothed-noise u0, f = 0, dt = 1/steps, tol 1e-8; `steps` chained CN steps
    through tfde_batch_cn_advance, then the same steps through a loop of
    single-problem tfde_cn_advance calls, both with the initial guess of
    `guess_order`.  Timed with CUDA events on the stream; inputs resident on
    the device."""
    import torch
    probs = inp.batched_instances(count=count, seed=4)
    dt = 1.0 / steps
    params = [T.make_params(p["n"], p["delta"], p["kp"], p["km"], dt) for p in probs]
    unknowns = sum(p["n"][0] * p["n"][1] * p["n"][2] for p in probs)
    u0 = [torch.from_numpy(inp.smoothed_uniform(tuple(reversed(p["n"])), 400 + i)).to(dev)
          for i, p in enumerate(probs)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": f"{count} problems, n in {{32,48,64,96,128}}, non-symmetric, {steps} CN steps, tol 1e-8",
           "unknowns": unknowns}
    out["initial_guess_order"] = guess_order
    B = T.tfde_batch_create(params, 20, stream)
    T.tfde_batch_set_guess_order(B, guess_order)

    def timed():
        us = [u.clone() for u in u0]
        T.tfde_batch_cn_advance(B, us, None, True, 1e-8, stream)    # warm-up step (restarts the chain)
        us = [u.clone() for u in u0]
        torch.cuda.synchronize()
        e0.record(stream)
        iters = 0
        for m in range(steps):
            infos = T.tfde_batch_cn_advance(B, us, None, m == 0, 1e-8, stream)
            iters += sum(i.iters for i in infos)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        return {"problem_steps_per_s": count * steps / sec, "unknown_steps_per_s": unknowns * steps / sec,
                "ms_per_step": 1e3 * sec / steps, "iters_per_problem_step": iters / (count * steps)}

    try:
        T.tfde_tune_clear()
        out["batched_default_launches"] = timed()
        # the autotuner on the batch's grouped launch classes, then the same steps
        t0 = time.perf_counter()
        T.tfde_batch_tune(B, 10, stream)
        table = T.tfde_tune_get()
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        out["autotuner"] = {"seconds": time.perf_counter() - t0, "classes": len(table),
                            "changed": sum(1 for e in table if (e["grid"], e["stages"]) != (min(e["tiles"], sms), 2)),
                            "trial_us_default": sum(e["us_default"] for e in table),
                            "trial_us_tuned": sum(e["us"] for e in table), "table": table}
        out["batched"] = timed()
        # the defaults once more (interleaved, so that drift between runs shows)
        T.tfde_tune_clear()
        again = timed()
        # the same cycles in the grid basis (five operator and six
        # preconditioner passes per Arnoldi step instead of three)
        T.tfde_batch_set_spectral_inner(B, False)
        out["grid_basis_default_launches"] = timed()
        T.tfde_batch_set_spectral_inner(B, True)
        d0 = out["batched_default_launches"]["problem_steps_per_s"]
        out["batched_default_launches"]["problem_steps_per_s_again"] = again["problem_steps_per_s"]
        out["tuned_vs_default"] = out["batched"]["problem_steps_per_s"] / (0.5 * (d0 + again["problem_steps_per_s"]))
    finally:
        T.tfde_batch_destroy(B)
        T.tfde_tune_clear()
    hs = [T.tfde_assemble(p, T.TFDE_MIXED, stream) for p in params]
    for h in hs:
        T.tfde_set_guess_order(h, guess_order)
    try:
        us = [u.clone() for u in u0]
        for i, h in enumerate(hs):
            T.tfde_cn_advance(h, us[i], None, True, 1e-8, stream)   # warm-up
        us = [u.clone() for u in u0]
        torch.cuda.synchronize()
        e0.record(stream)
        iters = 0
        for m in range(steps):
            for i, h in enumerate(hs):
                iters += T.tfde_cn_advance(h, us[i], None, m == 0, 1e-8, stream).iters
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        out["loop_of_single_calls"] = {"problem_steps_per_s": count * steps / sec,
                                       "unknown_steps_per_s": unknowns * steps / sec,
                                       "iters_per_problem_step": iters / (count * steps)}
    finally:
        for h in hs:
            T.tfde_destroy(h)
    out["speedup_vs_loop"] = out["batched"]["problem_steps_per_s"] / out["loop_of_single_calls"]["problem_steps_per_s"]
    # the symmetric variant of the same problems (k- = k+): the batched PCG
    # against every problem through the batched GMRES cycles
    sym_params = [T.make_params(p["n"], p["delta"], p["kp"], p["kp"], dt) for p in probs]
    B = T.tfde_batch_create(sym_params, 20, stream)
    T.tfde_batch_set_guess_order(B, guess_order)
    try:
        sym = {"workload": f"the same {count} problems with k- = k+ (symmetric), {steps} CN steps, tol 1e-8"}
        for key, pcg in (("pcg", True), ("gmres", False)):
            T.tfde_batch_set_symmetric_pcg(B, pcg)
            sym[key] = timed()
        sym["pcg_solves"] = T.tfde_batch_pcg_solves(B)
        sym["pcg_vs_gmres"] = sym["pcg"]["problem_steps_per_s"] / sym["gmres"]["problem_steps_per_s"]
        out["symmetric_variant"] = sym
    finally:
        T.tfde_batch_destroy(B)
    return out


# ----------------------------------------------------------- reference arm
def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    W = inp.WORKLOADS[WORKLOAD]
    n = args.n or W["n"]
    dt = 1.0 / W["M"]
    # warm-up steps untimed, then timed steps, all bounded by a few minutes
    budget = 180.0
    t0 = time.perf_counter()
    oracle_steps(n, W["delta"], W["kp"], dt, W["tol"], 0.0, max_steps=max(1, min(args.warmup, 1)))
    per = time.perf_counter() - t0
    k = max(1, min(args.steps, int(budget / max(per, 1e-9))))
    steps, sec = oracle_steps(n, W["delta"], W["kp"], dt, W["tol"], 1e30, max_steps=k)
    value = steps / sec
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": 1, "ms_per_step": 1e3 * sec / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**workload_config(n, W, dt, W["tol"]), "solver": "oracle PCG(tau), FP64, x0 = u^(m-1)"},
            "cpu_baseline": {"kind": "oracle", "cores": cpu_cores(), "value": value, "unit": UNIT,
                             "sample": f"{steps} CN step(s) of the n={n} workload (numpy FP64 oracle)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
