#!/usr/bin/env python
"""Benchmark of the RIOT inner loop on one GB300 (and N independent replicas).

Workload: Lorenz-96, n = 4096, F = 8, dt = 0.05, 200-step window, 25% of the
variables observed at fixed random indices every 4 steps (51 200
observations, sigma_o = 1), Gaussian B (sigma_b = 1, length 4), k = 512
Gaussian sketch columns, q = 1 power iteration.  A step is one full inner
loop: sketch draw, 2 x 512 Hessian-vector products (tangent-linear +
adjoint integrations), CholeskyQR, the projected matrix K, its FP64
tridiagonal eigendecomposition, the Ritz vectors and the adaptive increment.
The outer-loop prerequisites (nonlinear trajectory, gradient) run once before
the timed region.  The same line carries the Hessian-vector products of the
tracer-transport inversion on its full 192 x 192 x 30 grid (bc_transport).

Metric: Hessian-vector products per second of inner-loop wall time (with the
inner-loop milliseconds), for the mixed-precision path and the plain FP64
GPU form of the same algorithm.  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import advdiff as bc_synth  # noqa: E402
from synth import configs  # noqa: E402

WORKLOAD = "l96_n4096_F8_T200_obs25pct_every4_k512_q1"
import hashlib
import re

# DRAM bytes (read + write) of the dominant kernels come from the ncu summaries under
# profiles/ (one 512-column Hessian launch of the workload above; one RK4 step of 32 tracer
# columns on the 192 x 192 x 30 grid).  Each summary records the sha256 of the kernel's
# source file at capture time; a summary whose source has changed since is stale and the
# bench reports traffic null instead of an old number.
PROFILES = os.path.join(ROOT, "profiles")
KERNEL_SOURCES = os.path.join(ROOT, "paper_1906_01413_gb300", "csrc")


def profiled_traffic(summary, source):
    """(bytes per unit, capture note) from a profiles/ summary, or (None, why) when stale."""
    try:
        text = open(os.path.join(PROFILES, summary)).read()
        want = hashlib.sha256(open(os.path.join(KERNEL_SOURCES, source), "rb").read()).hexdigest()
    except OSError as e:
        return None, "no summary: %s" % e
    h = re.search(r"source sha256: ([0-9a-f]{64})", text)
    b = re.search(r"dram bytes per unit: ([0-9.eE+]+)", text)
    if not h or not b:
        return None, "summary %s has no source hash or byte count" % summary
    if h.group(1) != want:
        return None, "stale: %s changed since the capture in %s" % (source, summary)
    return float(b.group(1)), summary
METRIC = "RIOT inner-loop Hessian-vector products per second (inner-loop wall time)"
UNIT = "HVP/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="riot", choices=["riot", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-bc", action="store_true", help="skip the tracer-transport Hessian products")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch of 96 windows")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned sketch proposal leg")
    ap.add_argument("--learned-windows", type=int, default=64,
                    help="training windows of the learned sketch leg (the workload names 2000: about 3 minutes "
                         "of data generation)")
    ap.add_argument("--learned-steps", type=int, default=500, help="training steps (batches of 8 windows)")
    ap.add_argument("--no-precond", action="store_true", help="skip the preconditioned inner-loop leg")
    ap.add_argument("--no-deflated", action="store_true", help="skip the deflated multi-level mixed-precision leg")
    ap.add_argument("--no-comparators", action="store_true",
                    help="skip the paper's other inner loops (Algorithms 1, 2 and 4) on the same window")
    ap.add_argument("--clock-log", default=None,
                    help="CSV of the nvidia-smi clock samples taken during the timed steps (%%d: rank); "
                         "default: a file in the temporary directory")
    ap.add_argument("--hvp-kernel", choices=["cta_barrier", "warp_pairs", "warp_shuffle", "cta_two_per_sm"],
                    default="cta_barrier",
                    help="FP32 Hessian kernel of --only hvp")
    ap.add_argument("--only", choices=["bc", "batch", "learned", "varcg", "varbl", "psas", "hvp"], default=None,
                    help="run one secondary leg alone and print its JSON (profiling)")
    ap.add_argument("--bc-cols", type=int, default=128, help="sketch columns per tracer Hessian call")
    ap.add_argument("--profile", action="store_true",
                    help="bracket the first timed step with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_value(ms_local, units_per_step, world, pg=None, device=None):
    """Whole-job step time and throughput over independent replicas: the step time is the
    maximum over ranks, and every rank processed units_per_step per step."""
    ms = float(ms_local)
    if pg is not None and world > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_step / (ms * 1e-3)


def band_width(n, ell):
    """Number of taps of the banded Gaussian square-root kernel (same rule as the library)."""
    d = np.arange(n, dtype=np.float64)
    reach = int(math.ceil(40.0 * ell / n)) + 1
    row = sum(np.exp(-((d + j * n) ** 2) / (ell * ell)) for j in range(-reach, reach + 1))
    row = row / np.sqrt(np.sum(row * row))
    h = 0
    for dd in range(1, n // 2 + 1):
        if abs(row[dd]) > 1e-18 * row[0]:
            h = dd
    return n if 2 * h + 1 >= n else 2 * h + 1


def hvp_flops(n, T, p, taps):
    """Algorithmic FLOPs of one Hessian-vector product (FMA = 2):
    TL RK4 step 33 n, AD RK4 step 34 n, L and L^T band 2 * 2 * taps * n,
    observation scaling and scatter 3 per observation."""
    return 67.0 * n * T + 4.0 * taps * n + 3.0 * p


class ClockSampler:
    def __init__(self, path, index):
        self.path = path
        self.proc = None
        self.index = index

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return self
        # the timed region starts only once the first sample is on file (bounded wait)
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0:
            try:
                if os.path.getsize(self.path) > 0:
                    break
            except OSError:
                pass
            time.sleep(0.01)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [l.split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def build_problem(R, torch, cfg, dev, precision, kmax):
    from paper_1906_01413_gb300 import workloads
    return workloads.l96_twin(R, torch, cfg, dev, precision, kmax)


def time_inner_loop(R, torch, ctx, cfg, steps, warmup, flush, dv, profile=False, k=None):
    """Per-step CUDA-event times of riot_rsvd + riot_increment (L2 flushed between steps)."""
    k = cfg.k if k is None else k
    s = torch.cuda.current_stream()
    times, phases = [], []
    for i in range(warmup + steps):
        flush.zero_()
        torch.cuda.synchronize()
        prof = profile and i == warmup
        if prof:
            torch.cuda.profiler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        lam = R.riot_rsvd(ctx.h, k, cfg.q, sketch_stream=configs.STREAM_SKETCH0)
        mode = R.riot_increment(ctx.h, dv)
        e1.record(s)
        torch.cuda.synchronize()
        if prof:
            torch.cuda.profiler.stop()
        if i >= warmup:
            times.append(e0.elapsed_time(e1))
            ph = R.riot_rsvd_timings(ctx.h)
            ph["jacobi_sweeps"] = R.riot_rsvd_sweeps(ctx.h)
            phases.append(ph)
    return times, phases, lam, mode


DEFLATED_LEVELS = (256, 320)


def bench_deflated(R, torch, cfg, dev, flush, warmup, steps, levels=DEFLATED_LEVELS):
    """The deflated multi-level mixed-precision eigendecomposition (riot_rsvd_deflated) plus the
    increment on the same window: per-step CUDA-event times, the cost reduction of its increment
    (Eq. 3 in FP64) and its pairs."""
    kmax = sum(levels)
    ctx, xb, _ = build_problem(R, torch, cfg, dev, R.RIOT_PREC_MIXED, kmax)
    R.riot_outer_begin(ctx.h, xb)
    dv = torch.empty(cfg.n, dtype=torch.float64, device=dev)
    s = torch.cuda.current_stream()
    times = []
    for i in range(warmup + steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        lam = R.riot_rsvd_deflated(ctx.h, list(levels), cfg.q, 0.0, configs.STREAM_SKETCH0, kmax=kmax)
        mode = R.riot_increment(ctx.h, dv)
        e1.record(s)
        torch.cuda.synchronize()
        if i >= warmup:
            times.append(e0.elapsed_time(e1))
    red = R.riot_quadratic_cost(ctx.h) - R.riot_quadratic_cost(ctx.h, dv)
    ph = R.riot_rsvd_timings(ctx.h)
    ctx.close()
    ms = statistics.mean(times)
    hvps = (cfg.q + 1) * sum(levels)
    return {"what": "riot_rsvd_deflated: levels of %s columns, q = %d, each on the operator deflated by the "
                    "pairs kept before (FP32 products, two-pass FP32 projections), then riot_increment"
                    % (list(levels), cfg.q),
            "ms_per_step": ms, "hvps_per_step": hvps, "value": hvps / (ms * 1e-3), "unit": UNIT,
            "pairs": int(lam.size), "mode": int(mode), "lambda1": float(lam[0]), "lambda_min": float(lam[-1]),
            "cost_reduction": red, "phases_ms": ph}


def bench_precond(R, torch, ctx, xb, cfg, flush, dv, warmup, steps, plain_ms):
    """Algorithm 3 with precond = rotation = true on the same window: outer loop 1 from the
    background (the timed steps above moved x without re-linearising), its pairs with positive
    eigenvalue become the factor P'_1 (riot_precond_push), then timed preconditioned inner loops:
    riot_rsvd of A_2 = P_2^T (I + A) P_2 - I on a rotated sketch and riot_increment mapped by P_2.
    Loop 2 is linearised at the background again: one full step on this 200-step window leaves
    the attractor (the LRU step applies the unresolved part of a gradient grown by the
    tangent-linear model unscaled), and the inner-loop cost does not depend on the state."""
    R.riot_outer_begin(ctx.h, xb, torch.zeros_like(xb))
    lam = R.riot_rsvd(ctx.h, cfg.k, cfg.q, sketch_stream=configs.STREAM_SKETCH0)
    R.riot_increment(ctx.h, dv)
    m = int(np.sum(lam > 0))
    R.riot_precond_enable(ctx.h, m, True)
    t0 = time.perf_counter()
    R.riot_precond_push(ctx.h, m)
    push_s = time.perf_counter() - t0
    R.riot_outer_begin(ctx.h, xb, torch.zeros_like(xb))
    times, phases, lam2, mode = time_inner_loop(R, torch, ctx, cfg, steps, warmup, flush, dv)
    R.riot_precond_enable(ctx.h, 0, False)
    ms = statistics.mean(times)
    ph = {key: statistics.mean(p_[key] for p_ in phases) for key in phases[0]}
    return {"what": "inner loop of Algorithm 3 with precond = rotation = true (one factor of %d pairs)" % m,
            "ms_per_step": ms, "value": (cfg.q + 1) * cfg.k / (ms * 1e-3), "unit": UNIT,
            "overhead_vs_plain": ms / plain_ms - 1.0, "phases_ms": ph, "push_ms": push_s * 1e3,
            "lambda1": float(lam2[0]), "mode": int(mode)}


def bench_comparator(R, torch, dev, flush, which, warmup, steps):
    """The paper's other inner loops on the large Lorenz-96 window (mixed-precision context):
    varcg = Algorithm 1 with m = 64 (one Hessian product per iteration, sequential);
    varbl = Algorithm 2 with l = 64 samples and m = 8 block steps (512 products; the starting
    block is the gradient plus Gaussian columns: its content does not change the cost);
    psas = Algorithm 4 with m = 512 sketch columns and q = 1 in observation space (p = 51 200).
    Each step is one call, timed with CUDA events after an L2 flush."""
    cfg = configs.l96_large()
    ctx, xb, p = build_problem(R, torch, cfg, dev, R.RIOT_PREC_MIXED, cfg.k)
    R.riot_outer_begin(ctx.h, xb)
    s = torch.cuda.current_stream()
    n = cfg.n
    if which == "varbl":
        l, m = 64, 8
        g = torch.empty(n, dtype=torch.float64, device=dev)
        R.riot_get_state(ctx.h, g=g)
        B0 = g[None, :] + torch.randn(l, n, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(7)) \
            * g.abs().mean()
        B0 = B0.contiguous()
    times, info = [], {}
    dv = torch.empty(n, dtype=torch.float64, device=dev)
    for i in range(warmup + steps):
        if which == "psas" and i:
            R.riot_outer_begin(ctx.h, xb, torch.zeros_like(xb))
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        if which == "varcg":
            theta, used = R.riot_varcg(ctx.h, 64, dv)
            info = {"m": used, "hvps": used, "theta1": float(theta.max())}
        elif which == "varbl":
            theta, nb = R.riot_varbl(ctx.h, l, m, B0, dv)
            info = {"l": l, "m": nb, "hvps": l * nb, "theta1": float(theta[0])}
        else:
            lam, mode = R.riot_psas(ctx.h, 512, 1, sketch_stream=configs.STREAM_SKETCH0, dv=dv)
            info = {"m": 512, "q": 1, "p": int(p), "dual_products": 2 * 512, "lambda1": float(lam[0]), "mode": mode}
        e1.record(s)
        torch.cuda.synchronize()
        if i >= warmup:
            times.append(e0.elapsed_time(e1))
    # cost reduction J~(0) - J~(dv) of the leg's increment (Eq. 3, FP64)
    red = R.riot_quadratic_cost(ctx.h) - R.riot_quadratic_cost(ctx.h, dv)
    ctx.close()
    ms = statistics.mean(times)
    units = info.get("hvps", info.get("dual_products", 0))
    return {"leg": which, "workload": WORKLOAD, "ms_per_call": ms, "products_per_s": units / (ms * 1e-3),
            "cost_reduction": red, **info}


def bench_hvp(R, torch, dev, flush, kernel, warmup, steps):
    """512 Hessian-vector products of the large Lorenz-96 window in one riot_hessian_apply (the
    inner loop's dominant launch), timed alone with CUDA events after an L2 flush."""
    cfg = configs.l96_large()
    ctx, xb, p = build_problem(R, torch, cfg, dev, R.RIOT_PREC_MIXED, cfg.k)
    R.riot_set_hvp_kernel(ctx.h, {"warp_pairs": R.RIOT_HVP_WARP_PAIRS, "warp_shuffle": R.RIOT_HVP_WARP_SHUFFLE,
                                  "cta_two_per_sm": R.RIOT_HVP_CTA_TWO_PER_SM}.get(kernel, R.RIOT_HVP_CTA_BARRIER))
    R.riot_outer_begin(ctx.h, xb)
    W = torch.empty(cfg.k, cfg.n, dtype=torch.float32, device=dev)
    R.riot_draw_normal(cfg.seed, configs.STREAM_SKETCH0, cfg.n, cfg.k, W)
    Y = torch.empty_like(W)
    s = torch.cuda.current_stream()
    times = []
    for i in range(warmup + steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        R.riot_hessian_apply(ctx.h, W, Y)
        e1.record(s)
        torch.cuda.synchronize()
        if i >= warmup:
            times.append(e0.elapsed_time(e1))
    ctx.close()
    ms = statistics.mean(times)
    flop = hvp_flops(cfg.n, cfg.T, p, band_width(cfg.n, cfg.ell)) * cfg.k
    return {"kernel": kernel, "workload": WORKLOAD, "ms_per_launch": ms, "tflops": flop / (ms * 1e-3) / 1e12,
            "hvps_per_launch": cfg.k}


def build_bc_problem(R, torch, cfg, dev, precision, kmax):
    from paper_1906_01413_gb300 import workloads
    return workloads.bc_twin(R, torch, cfg, dev, precision, kmax)


def bench_bc_transport(R, torch, dev, flush, hbm_peak, ncols=128, reps=2):
    """Hessian-vector products of the tracer inversion on its full grid
    (192 x 192 x 30 cells, 240 steps, 8000 observations), one launch block of
    ncols sketch columns per call, FP32 transport."""
    cfg = bc_synth.bc_large()
    ctx, xb, p = build_bc_problem(R, torch, cfg, dev, R.RIOT_PREC_MIXED, ncols)
    R.riot_outer_begin(ctx.h, xb)
    W = torch.empty(ncols, cfg.n, dtype=torch.float32, device=dev)
    R.riot_draw_normal(cfg.seed, bc_synth.STREAM_SKETCH0, cfg.n, ncols, W)
    Y = torch.empty_like(W)
    R.riot_hessian_apply(ctx.h, W, Y)
    s = torch.cuda.current_stream()
    times = []
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        R.riot_hessian_apply(ctx.h, W, Y)
        e1.record(s)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ctx.close()
    ms = statistics.mean(times)
    ncells = cfg.nx * cfg.ny * cfg.nz
    bytes_per_hvp = 8.0 * ncells * cfg.T * 2
    # measured DRAM bytes of one step of one column, times the 2T steps of a product
    step_bytes, bc_note = profiled_traffic("adv_step_f2_kernel_bc_192x192x30_P32.md", "advdiff.cu")
    bc_traffic = None if step_bytes is None else step_bytes * 2 * cfg.T
    achieved = bytes_per_hvp * ncols / (ms * 1e-3) / 1e9
    return {"workload": "bc_%dx%dx%d_T%d_obs%d_blocks%d" % (cfg.nx, cfg.ny, cfg.nz, cfg.T, p, cfg.nblocks),
            "value": ncols / (ms * 1e-3), "unit": "HVP/s", "ms_per_hvp": ms / ncols, "columns_per_call": ncols,
            "dtype": "f32",
            "roofline": {"bound": "hbm", "kernel": "adv_step_f2_kernel<15,32,8> (whole product timed)",
                         "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                         "traffic": bc_traffic, "traffic_source": bc_note, "bytes_per_hvp": bytes_per_hvp,
                         "bytes_basis": "one FP32 read and write of the tracer per RK4 step, TL and AD"}}


def bench_bc_inner_loop(R, torch, dev, flush):
    """One RIOT inner loop of the tracer inversion on its full grid (Algorithm 3 with k = 1024,
    q = 1: 2048 Hessian-vector products, CholeskyQR, K, the 1024 x 1024 FP64 eigensolver, Ritz
    vectors, increment), mixed precision, timed once with CUDA events after an L2 flush (one
    inner loop is about 2048 x 6.7 ms of products)."""
    cfg = bc_synth.bc_large()
    ctx, xb, p = build_bc_problem(R, torch, cfg, dev, R.RIOT_PREC_MIXED, cfg.k)
    R.riot_outer_begin(ctx.h, xb)
    dv = torch.empty(cfg.n, dtype=torch.float64, device=dev)
    s = torch.cuda.current_stream()
    flush.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    lam = R.riot_rsvd(ctx.h, cfg.k, cfg.q, sketch_stream=bc_synth.STREAM_SKETCH0)
    mode = R.riot_increment(ctx.h, dv)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ph = R.riot_rsvd_timings(ctx.h)
    red = R.riot_quadratic_cost(ctx.h) - R.riot_quadratic_cost(ctx.h, dv)
    pairs = R.riot_increment_pairs(ctx.h)
    ctx.close()
    hvps = (cfg.q + 1) * cfg.k
    return {"workload": "bc_%dx%dx%d_T%d_obs%d_blocks%d_k%d_q%d" % (cfg.nx, cfg.ny, cfg.nz, cfg.T, p, cfg.nblocks,
                                                                  cfg.k, cfg.q),
            "inner_loop_ms": ms, "hvps_per_step": hvps, "value": hvps / (ms * 1e-3), "unit": "HVP/s",
            "phases_ms": ph, "lambda1": float(lam[0]), "lambda_k": float(lam[-1]), "mode": int(mode),
            "pairs_retained": pairs, "cost_reduction": red, "steps_timed": 1}


def bench_batch(R, torch, dev, warmup, steps, fp64_baseline=True):
    """96 independent Lorenz-96 windows of uneven n, T and k: one inner loop
    of every window per step, batched (persistent Hessian launches, one CUDA
    graph, autotuned launch shape) against the same windows one at a time
    (mixed precision, and the plain FP64 form)."""
    from paper_1906_01413_gb300 import workloads
    wins = configs.batch_windows()
    q = 1
    hvps = sum((q + 1) * w.k for w in wins)
    s = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    ctxs = []
    for w in wins:
        ctx, xb, _ = workloads.l96_twin(R, torch, w, dev, R.RIOT_PREC_MIXED, w.k)
        R.riot_outer_begin(ctx.h, xb)
        ctxs.append(ctx)
    b = R.riot_batch_create([c.h for c in ctxs], [w.k for w in wins], q)
    P, S, tune_ms = R.riot_batch_autotune(b)
    launches0 = R.riot_kernel_launches()
    statuses = None
    for _ in range(warmup):
        statuses = R.riot_batch_run(b, len(wins), sketch_stream=configs.STREAM_SKETCH0, use_graph=True, check=False)
    l1 = R.riot_kernel_launches()
    times = [timed(lambda: R.riot_batch_run(b, len(wins), sketch_stream=configs.STREAM_SKETCH0, use_graph=True,
                                            check=False))
             for _ in range(steps)]
    graph_launches = R.riot_kernel_launches() - l1    # host-issued launches while replaying: 0 expected
    batched_ms = statistics.mean(times)
    eager_ms = timed(lambda: R.riot_batch_run(b, len(wins), sketch_stream=configs.STREAM_SKETCH0, use_graph=False,
                                              check=False))
    hvp_ms = timed(lambda: R.riot_batch_hessian_apply(b))
    R.riot_batch_destroy(b)

    alone_failed = []

    def one_at_a_time(cs):
        for i, (w, c) in enumerate(zip(wins, cs)):
            try:
                R.riot_rsvd(c.h, w.k, q, sketch_stream=configs.STREAM_SKETCH0)
                R.riot_increment(c.h)
            except R.RiotError:
                alone_failed.append(i)

    alone_ms = timed(lambda: one_at_a_time(ctxs))
    for c in ctxs:
        c.close()
    out = {"workload": "l96_batch%d_n%d-%d_T%d-%d_k%d-%d_q%d" % (
               len(wins), min(w.n for w in wins), max(w.n for w in wins), min(w.T for w in wins),
               max(w.T for w in wins), min(w.k for w in wins), max(w.k for w in wins), q),
           "windows": len(wins), "hvps_per_step": hvps, "value": hvps / (batched_ms * 1e-3), "unit": "HVP/s",
           "ms_per_step": batched_ms, "graph": True, "batched_eager_ms": eager_ms,
           "batched_hvp_launch_ms": hvp_ms, "one_at_a_time_mixed_ms": alone_ms,
           "speedup_vs_one_at_a_time_mixed": alone_ms / batched_ms,
           "autotune": {"probes_cap": P, "ring_depth": S, "hvp_launch_ms": tune_ms},
           "host_launches_per_graph_step": int(graph_launches) // max(1, steps),
           "windows_failed": [i for i, st in enumerate(statuses or []) if st != 0],
           "one_at_a_time_mixed_windows_failed": alone_failed}
    if fp64_baseline:
        tot = 0.0
        fp64_failed = []
        for i, w in enumerate(wins):
            c, xb, _ = workloads.l96_twin(R, torch, w, dev, R.RIOT_PREC_FP64, w.k)
            R.riot_outer_begin(c.h, xb)

            def run64():
                try:
                    R.riot_rsvd(c.h, w.k, q, sketch_stream=configs.STREAM_SKETCH0)
                    R.riot_increment(c.h)
                except R.RiotError:
                    fp64_failed.append(i)

            tot += timed(run64)
            c.close()
        out["one_at_a_time_fp64_ms"] = tot
        out["one_at_a_time_fp64_windows_failed"] = fp64_failed
        out["speedup_vs_one_at_a_time_fp64"] = tot / batched_ms
    return out


def bench_learned_sketch(R, torch, dev, n_train=64, n_test=8, steps=500):
    """Learned sketch proposal on Lorenz-96 n=4096, F=12, T=300 windows: a
    periodic conv-net (4 layers, 64 channels, 8 input snapshots, 128
    directions) trained on the leading 128 eigenvectors that riot_rsvd (k=512
    Gaussian, q=1) produced on n_train windows, then used on n_test unseen
    windows as [128 proposed | k - 128 Gaussian] sketches, gated by the
    Rayleigh residual (rho <= 1e-2, else pure Gaussian).  Reports the cost
    reduction of the resulting increments against Gaussian sketches."""
    from paper_1906_01413_gb300 import workloads
    n, T, m, C, width = 4096, 300, 128, 8, 64
    ks = [128, 256, 384, 512]

    def wcfg(w):
        # the workload gives no step length: the paper's Lorenz-96 step dt = 0.01 (Section 3.1)
        return configs.L96Config(name="ls%d" % w, n=n, F=12.0, dt=0.01, T=T, obs_every=4, obs_frac=0.25,
                                 obs_layout="random", ell=4.0, k=512, q=1, seed=configs.BASE_SEED + 5000 + w)

    def window(w):
        cfg = wcfg(w)
        ctx, xb, _ = workloads.l96_twin(R, torch, cfg, dev, R.RIOT_PREC_MIXED, 512)
        R.riot_outer_begin(ctx.h, xb)
        traj = torch.empty(T + 1, n, dtype=torch.float64, device=dev)
        R.riot_get_trajectory(ctx.h, traj)
        x = torch.empty(C, n, dtype=torch.float32, device=dev)
        R.riot_sketchnet_input(traj, T, n, C, x)
        return ctx, x

    t0 = time.perf_counter()
    xs, Us = [], []
    for w in range(n_train):
        ctx, x = window(w)
        R.riot_rsvd(ctx.h, 512, 1, sketch_stream=configs.STREAM_SKETCH0)
        U = torch.empty(512, n, dtype=torch.float64, device=dev)
        R.riot_get_state(ctx.h, U=U)
        xs.append(x)
        Us.append(U[:m].float())
        ctx.close()
    X = torch.stack(xs).contiguous()
    Ut = torch.stack(Us).contiguous()
    data_s = time.perf_counter() - t0
    from synth import learned
    flat = torch.tensor(learned.initial_params(C, width, m).astype(np.float32), device=dev)
    net = R.riot_sketchnet_create(C, width, m, n_max=n, batch_max=8, r_max=m)
    R.riot_sketchnet_set_params(net, flat)
    rng = np.random.default_rng(1)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    losses = []
    for it in range(steps):
        idx = torch.tensor(rng.choice(n_train, 8, replace=False), device=dev)
        losses.append(R.riot_sketchnet_train_step(net, X[idx].contiguous(), Ut[idx].contiguous(), 0.1, 2e-3))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1

    def dJ(ctx64, dv):
        # reduction of the quadratic inner cost, -(g.dv + |dv|^2/2 + dv.A dv/2), with an FP64
        # product (these windows' Hessians exceed the FP32 range)
        g = torch.empty(n, dtype=torch.float64, device=dev)
        R.riot_get_state(ctx64.h, g=g)
        w = dv.reshape(1, n).contiguous()
        Aw = torch.empty_like(w)
        R.riot_hessian_apply(ctx64.h, w, Aw)
        return -float(g @ dv + 0.5 * dv @ dv + 0.5 * dv @ Aw[0])

    rows = {"gauss": {k: [] for k in ks}, "proposal_gated": {k: [] for k in ks[1:]},
            "proposal_ungated": {k: [] for k in ks[1:]}}
    rhos, used = [], []
    capture = []
    for w in range(n_test):
        ctx, x = window(10000 + w)
        ctx64, xb64, _ = workloads.l96_twin(R, torch, wcfg(10000 + w), dev, R.RIOT_PREC_FP64, 1)
        R.riot_outer_begin(ctx64.h, xb64)
        Z = torch.empty(1, m, n, dtype=torch.float32, device=dev)
        R.riot_sketchnet_forward(net, x.reshape(1, C, n).contiguous(), Z, bf16=True)
        P = Z[0].contiguous()
        dv = torch.empty(n, dtype=torch.float64, device=dev)
        for k in ks:
            R.riot_rsvd(ctx.h, k, 1, sketch_stream=configs.STREAM_SKETCH0)
            if k == 512:
                U = torch.empty(512, n, dtype=torch.float64, device=dev)
                R.riot_get_state(ctx.h, U=U)
                Q, _ = torch.linalg.qr(P.double().T)
                capture.append(float((U[:m] @ Q).pow(2).sum()) / m)
            R.riot_increment(ctx.h, dv)
            rows["gauss"][k].append(dJ(ctx64, dv))
        for k in ks[1:]:
            _, rho, u = R.riot_rsvd_proposal(ctx.h, k, 1, P, m, rho_max=1e-2, sketch_stream=configs.STREAM_SKETCH0)
            R.riot_increment(ctx.h, dv)
            rows["proposal_gated"][k].append(dJ(ctx64, dv))
            if k == 256:
                rhos.append(rho)
                used.append(u)
            R.riot_rsvd_proposal(ctx.h, k, 1, P, m, rho_max=1e30, sketch_stream=configs.STREAM_SKETCH0)
            R.riot_increment(ctx.h, dv)
            rows["proposal_ungated"][k].append(dJ(ctx64, dv))
        ctx.close()
        ctx64.close()
    R.riot_sketchnet_destroy(net)
    mean = {key: {k: float(np.mean(v)) for k, v in d.items()} for key, d in rows.items()}
    target = mean["gauss"][512]

    def k_needed(d):
        for k in sorted(d):
            if d[k] >= target * (1 - 1e-3):
                return k
        return None

    return {"workload": "l96_n4096_F12_dt0.01_T300_obs25pct_every4_proposal128", "train_windows": n_train,
            "test_windows": n_test, "train_steps": steps, "net": "4 periodic conv layers, 64 channels, kernel 5, "
            "8 snapshots -> 128 directions, FP32 training, BF16 inference",
            "data_s": data_s, "train_s": train_s, "loss_first": losses[0], "loss_last": losses[-1],
            "held_out_capture_of_leading_128": float(np.mean(capture)), "random_capture": m / n,
            "rho_at_k256": rhos, "proposal_used_at_k256": used,
            "mean_cost_reduction": {key: {str(k): v for k, v in d.items()} for key, d in mean.items()},
            "k_for_gauss512_reduction": {"gauss": k_needed(mean["gauss"]),
                                         "proposal_gated": k_needed(mean["proposal_gated"]),
                                         "proposal_ungated": k_needed(mean["proposal_ungated"])}}


def _oracle_worker(root, workload, seconds, seed, barrier, out):
    """One process of the CPU baseline: build the workload, wait for the others (so that all
    time the same interval), run FP64 oracle Hessian-vector products for `seconds`."""
    if root not in sys.path:
        sys.path.insert(0, root)
    from oracle import problem, riot as orc
    from synth import configs as cf
    cfg = getattr(cf, workload)()
    prob = problem.build(cfg)
    traj = orc.trajectory(prob, prob.x_b)
    rng = np.random.default_rng(seed)
    try:
        barrier.wait(timeout=600)
    except Exception:
        out.put((0, 0.0))
        return
    t0 = time.perf_counter()
    done = 0
    while True:
        orc.hvp(prob, traj, rng.standard_normal((cfg.n, 1)))
        done += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    out.put((done, el))


def _collect(out, procs, count, limit_s):
    """`count` results from the workers' queue; stops early (terminating the workers this
    process started) when one of them exits with an error or the time limit passes."""
    import queue
    res, deadline = [], time.time() + limit_s
    while len(res) < count:
        try:
            res.append(out.get(timeout=5))
        except queue.Empty:
            if any(pr.exitcode not in (None, 0) for pr in procs) or time.time() > deadline:
                for pr in procs:
                    if pr.is_alive():
                        pr.terminate()
                raise RuntimeError("a CPU oracle worker process failed or ran out of time")
    for pr in procs:
        pr.join(timeout=60)
    return res


def host_cores():
    """Cores this process may run on (the affinity set respects cpusets; cpu_count may not)."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_oracle_rate(seconds, workers, workload="l96_large"):
    """FP64 CPU oracle Hessian-vector products per second of the workload over `workers`
    spawned processes, each with one BLAS / OpenMP thread, timed together after a barrier.
    Returns (products, seconds, products per second)."""
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        barrier, out = ctx.Barrier(workers), ctx.Queue()
        procs = [ctx.Process(target=_oracle_worker, args=(ROOT, workload, seconds, 100 + w, barrier, out))
                 for w in range(workers)]
        for pr in procs:
            pr.start()
        res = _collect(out, procs, workers, 900)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    done = sum(d for d, _ in res)
    el = max(e for _, e in res)
    rate = sum(d / e for d, e in res if e > 0)
    return done, el, rate


def _reference_worker(root, workload, cols, nsteps, seed, barrier, out):
    """One process of the reference arm: per step, after a barrier with the other processes,
    `cols` FP64 oracle Hessian-vector products of the workload; reports each step's time."""
    if root not in sys.path:
        sys.path.insert(0, root)
    from oracle import problem, riot as orc
    from synth import configs as cf
    cfg = getattr(cf, workload)()
    prob = problem.build(cfg)
    traj = orc.trajectory(prob, prob.x_b)
    W = np.random.default_rng(seed).standard_normal((cfg.n, cols))
    for i in range(nsteps):
        try:
            barrier.wait(timeout=600)
        except Exception:
            out.put((i, -1.0))
            return
        t0 = time.perf_counter()
        orc.hvp(prob, traj, W)
        out.put((i, time.perf_counter() - t0))


def reference_arm(args):
    """The FP64 CPU oracle on the host cores: every step, each of nproc spawned processes (one
    BLAS thread each) computes `cols` Hessian-vector products of the workload; the step time is
    the slowest process's."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import multiprocessing as mp
    from oracle import _clib
    _clib.build()
    cfg = configs.l96_large()
    cores = host_cores()
    cols = 2
    nsteps = args.warmup + args.steps
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(cores), ctx.Queue()
    procs = [ctx.Process(target=_reference_worker, args=(ROOT, "l96_large", cols, nsteps, 200 + w, barrier, out))
             for w in range(cores)]
    for pr in procs:
        pr.start()
    step_max = [0.0] * nsteps
    for i, t in _collect(out, procs, cores * nsteps, 1800):
        if t < 0:
            raise RuntimeError("reference arm: a worker process failed to start its step")
        step_max[i] = max(step_max[i], t)
    per = statistics.mean(step_max[args.warmup:]) if args.steps > 0 else float("nan")
    value = cores * cols / per
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": cfg.n, "T": cfg.T, "k": cfg.k, "q": cfg.q},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d Hessian-vector products of the workload per step: %d per process on %d "
                                       "processes (FP64 C TL/AD + numpy L, one thread each)" % (cores * cols, cols,
                                                                                              cores)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    from paper_1906_01413_gb300 import riot as R
    rank, world, local = dist_env()
    R.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    if args.only:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        if args.profile:
            torch.cuda.profiler.start()
        if args.only == "learned":
            out = bench_learned_sketch(R, torch, dev, n_train=args.learned_windows, steps=args.learned_steps)
        elif args.only in ("varcg", "varbl", "psas"):
            out = bench_comparator(R, torch, dev, flush, args.only, args.warmup, max(1, args.steps))
        elif args.only == "hvp":
            out = bench_hvp(R, torch, dev, flush, args.hvp_kernel, args.warmup, max(1, args.steps))
        elif args.only == "bc":
            out = bench_bc_transport(R, torch, dev, flush, float(peaks.get("hbm_gbs", 6800.0)), ncols=args.bc_cols,
                                     reps=max(1, args.steps))
        else:
            out = bench_batch(R, torch, dev, args.warmup, max(1, args.steps), fp64_baseline=False)
        if args.profile:
            torch.cuda.profiler.stop()
        if rank == 0:
            print(json.dumps(out))
        return 0
    cfg = configs.l96_large()
    n, k, q, T = cfg.n, cfg.k, cfg.q, cfg.T

    # ---- mixed-precision path ------------------------------------------------------
    ctx, xb, p = build_problem(R, torch, cfg, dev, R.RIOT_PREC_MIXED, k)
    R.riot_outer_begin(ctx.h, xb)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    dv = torch.empty(n, dtype=torch.float64, device=dev)
    time_inner_loop(R, torch, ctx, cfg, 0, args.warmup, flush, dv)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    launches0 = R.riot_kernel_launches()
    wall0 = time.perf_counter()
    clock_log = (args.clock_log % rank) if args.clock_log and "%d" in args.clock_log else args.clock_log
    if not clock_log:
        import tempfile
        clock_log = os.path.join(tempfile.gettempdir(), "riot_bench_clocks_rank%d.csv" % rank)
    with ClockSampler(clock_log, local) as clk:
        times, phases, lam, mode = time_inner_loop(R, torch, ctx, cfg, args.steps, 0, flush, dv, args.profile)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = R.riot_kernel_launches() - launches0
    hvps_per_step = (q + 1) * k
    ms, value = job_value(statistics.mean(times), hvps_per_step, world, pg, dev)

    ph = {key: statistics.mean(p_[key] for p_ in phases) for key in phases[0]}
    hvp_launch_ms = ph["hvp"] / (q + 1)
    # cost reduction J~(0) - J~(dv) of the mixed increment (Eq. 3, FP64 tangent-linear pass)
    red_mixed = R.riot_quadratic_cost(ctx.h) - R.riot_quadratic_cost(ctx.h, dv)
    pairs_mixed = R.riot_increment_pairs(ctx.h)
    dv_mixed = dv.double().cpu().numpy().copy()
    taps = band_width(n, cfg.ell)
    flop_hvp = hvp_flops(n, T, p, taps)
    achieved = flop_hvp * k / (hvp_launch_ms * 1e-3) / 1e12
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    l96_traffic, l96_traffic_note = profiled_traffic("l96_hvp_tma_kernel_n4096_T200_k512.md", "l96_tma.cu")
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_nominal = sm_count * 128 * 2 * sm_max * 1e6 / 1e12
    try:   # FP32 / FP64 FMA throughput and FP64 latencies of this GPU, measured by the library
        alu = R.riot_measure_peaks(dev.index or 0)
    except R.RiotError as e:
        alu = {"error": str(e)}
    fp32_peak = alu.get("fp32_tflops", fp32_nominal)
    fp32_basis = ("measured: FP32 FMA throughput of riot_measure_peaks (8 independent chains per thread, "
                  "4 x 256 threads per SM), nominal %d SMs x 128 lanes x 2 x %.0f MHz = %.1f TFLOP/s"
                  % (sm_count, sm_max, fp32_nominal)) if "fp32_tflops" in alu else \
        "%d SMs x 128 FP32 lanes x 2 flop x %.0f MHz (max SM clock)" % (sm_count, sm_max)
    # FP64 work of the k x k chain (orth, K, eig) at algorithmic counts: 8 Cholesky factorisations
    # (k^3 / 3), M M^T (k^3) and N M^T (2 k^3), 4 triangular solves on k x k (k^3), the
    # tridiagonalisation and the accumulation of its Q (4/3 k^3 each), 2 eigenvector Grams (k^3)
    fp64_chain_flop = (8.0 / 3 + 3 + 4 + 8.0 / 3 + 2) * float(k) ** 3

    # ---- end to end through the C ABI with host buffers ------------------------------
    Om_host = torch.from_numpy(cfg.sketch(0).astype(np.float32)).pin_memory()
    Om_dev = torch.empty(k, n, dtype=torch.float32, device=dev)
    dv_host = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_times = []
    for i in range(args.warmup + max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Om_dev.copy_(Om_host, non_blocking=True)
        lam_e = R.riot_rsvd(ctx.h, k, q, Omega=Om_dev)
        R.riot_increment(ctx.h, dv)
        dv_host.copy_(dv, non_blocking=True)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    e2e_s = statistics.mean(e2e_times)
    precond = None
    if not args.no_precond:
        try:
            precond = bench_precond(R, torch, ctx, xb, cfg, flush, dv, 1, max(3, args.steps // 2), ms)
        except R.RiotError as e:   # keep the headline line; report the leg's failure in it
            precond = {"error": str(e)}

    # ---- tracer-transport inversion (workload 3): Hessian products on the full grid ----
    learned = None
    if not args.no_learned:
        learned = bench_learned_sketch(R, torch, dev, n_train=args.learned_windows, steps=args.learned_steps)
    batch = None
    if not args.no_batch:
        batch = bench_batch(R, torch, dev, args.warmup, max(3, args.steps // 3))
    comparators = None
    if not args.no_comparators:
        comparators = {}
        for which in ("varcg", "varbl", "psas"):
            try:
                comparators[which] = bench_comparator(R, torch, dev, flush, which, 1, 2)
            except R.RiotError as e:   # keep the headline line; report the leg's failure in it
                comparators[which] = {"error": str(e)}
    bc = None
    if not args.no_bc:
        bc = bench_bc_transport(R, torch, dev, flush, float(peaks.get("hbm_gbs", 6800.0)))
        try:
            bc["inner_loop"] = bench_bc_inner_loop(R, torch, dev, flush)
        except R.RiotError as e:   # keep the headline line; report the leg's failure in it
            bc["inner_loop"] = {"error": str(e)}

    # ---- deflated multi-level mixed precision (the same window) --------------------------
    deflated = None
    if not args.no_deflated:
        ctx.close()
        ctx = None
        deflated = bench_deflated(R, torch, cfg, dev, flush, 1, max(3, args.steps // 3))

    # ---- plain FP64 GPU form -----------------------------------------------------------
    fp64 = None
    if ctx is not None:
        ctx.close()
    if args.fp64_steps > 0:
        ctx64, xb64, _ = build_problem(R, torch, cfg, dev, R.RIOT_PREC_FP64, k)
        R.riot_outer_begin(ctx64.h, xb64)
        t64, ph64, lam64, mode64 = time_inner_loop(R, torch, ctx64, cfg, args.fp64_steps, 1, flush, dv)
        ms64 = statistics.mean(t64)
        red64 = R.riot_quadratic_cost(ctx64.h) - R.riot_quadratic_cost(ctx64.h, dv)
        dv64 = dv.double().cpu().numpy()
        lead = lam64 >= 2.0 ** -24 * lam64[0]
        fp64 = {"ms_per_step": ms64, "value": hvps_per_step / (ms64 * 1e-3), "unit": UNIT,
                "hvp_ms": statistics.mean(p_["hvp"] for p_ in ph64),
                "mode": int(mode64), "cost_reduction": red64,
                "speedup_of_mixed": ms64 / ms,
                "lambda1_rel_diff_mixed_vs_fp64": float(abs(lam[0] - lam64[0]) / abs(lam64[0])),
                "leading_lambda_rel_diff_mixed_vs_fp64": float(np.max(np.abs(lam[lead] - lam64[lead]) / lam64[lead])),
                "leading_lambdas": int(lead.sum()),
                "increment_rel_diff_mixed_vs_fp64": float(np.linalg.norm(dv_mixed - dv64) / np.linalg.norm(dv64)),
                "cost_reduction_rel_diff_mixed_vs_fp64": float(abs(red_mixed - red64) / abs(red64))}
        if deflated:
            # the FP64 form at the sketch size whose increment reaches the deflated path's reduction
            # (the reduction grows about linearly with k on this window: every pair adds a similar
            # share), to compare wall times at the same cost-function reduction
            target = deflated["cost_reduction"]
            k_eq = int(min(k, max(64, 8 * round(k * target / red64 / 8))))
            t_eq, _, _, _ = time_inner_loop(R, torch, ctx64, cfg, args.fp64_steps, 1, flush, dv, k=k_eq)
            red_eq = R.riot_quadratic_cost(ctx64.h) - R.riot_quadratic_cost(ctx64.h, dv)
            # one secant step between (k_eq, red_eq) and (k, red64) towards the target
            if k_eq < k and red64 != red_eq and abs(red_eq - target) > 0.005 * target:
                k2 = int(min(k, max(64, 8 * round((k_eq + (target - red_eq) * (k - k_eq) / (red64 - red_eq)) / 8))))
                if k2 != k_eq:
                    t2, _, _, _ = time_inner_loop(R, torch, ctx64, cfg, args.fp64_steps, 1, flush, dv, k=k2)
                    red2 = R.riot_quadratic_cost(ctx64.h) - R.riot_quadratic_cost(ctx64.h, dv)
                    if abs(red2 - target) < abs(red_eq - target):
                        k_eq, t_eq, red_eq = k2, t2, red2
        ctx64.close()
        fp64["equal_reduction"] = {
            "fp64": {"ms": ms64, "cost_reduction": red64},
            "mixed_plain": {"ms": ms, "cost_reduction": red_mixed, "pairs": pairs_mixed,
                            "reduction_ratio": red_mixed / red64},
        }
        if deflated:
            fp64["equal_reduction"]["mixed_deflated"] = {
                "ms": deflated["ms_per_step"], "cost_reduction": deflated["cost_reduction"],
                "pairs": deflated["pairs"], "reduction_ratio": deflated["cost_reduction"] / red64,
                "speedup_vs_fp64_k512": ms64 / deflated["ms_per_step"]}
            fp64["equal_reduction"]["fp64_at_equal_reduction"] = {
                "k": k_eq, "ms": statistics.mean(t_eq), "cost_reduction": red_eq,
                "deflated_mixed_speedup": statistics.mean(t_eq) / deflated["ms_per_step"],
                "deflated_reduction_over_this": deflated["cost_reduction"] / red_eq}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "T": T, "k": k, "q": q, "p_obs": int(p),
                       "precision": "TL/AD f32; CholeskyQR Grams exact on tensor cores (BF16 slices), Cholesky, tridiagonal eig, increment f64",
                       "l2": "256 MB buffer written between timed steps (flush)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "inner_loop_ms": ms},
            "phases_ms": ph,
            "roofline": {"bound": "alu", "kernel": "l96_hvp_tma_kernel<8,2,512>", "achieved": achieved,
                         "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                         "traffic": l96_traffic, "traffic_source": l96_traffic_note,
                         "peak_basis": fp32_basis,
                         "flop_per_hvp": flop_hvp, "hvp_per_launch": k, "launch_ms": hvp_launch_ms},
            "e2e": {"value": world * hvps_per_step / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(n * k * 4),
                    "d2h_bytes_per_step": int(n * 8 + k * 8)},
            "gpu_launches": int(launches),
            "wall_s_timed": wall}
    line["mixed_cost_reduction"] = {"value": red_mixed, "pairs_retained": pairs_mixed}
    chain_ms = ph["orth"] + ph["kmat"] + ph["eig"]
    line["fp64_chain"] = {
        "what": "the k x k FP64 linear algebra of the inner loop (CholeskyQR factorisations, K, eigensolver): "
                "latency-bound on this GPU (FP64 FMA latency and the serial pivots / reflectors)",
        "ms": chain_ms, "share_of_step": chain_ms / ms, "fp64_flop": fp64_chain_flop,
        "achieved_tflops": fp64_chain_flop / (chain_ms * 1e-3) / 1e12,
        "peak_tflops": alu.get("fp64_tflops"),
        "frac": (fp64_chain_flop / (chain_ms * 1e-3) / 1e12 / alu["fp64_tflops"]) if "fp64_tflops" in alu else None,
        "measured_alu": alu}
    if comparators:
        line["paper_comparison"] = {
            "what": "the paper's inner loops on the same window, each one call after an L2 flush: RIOT "
                    "(Algorithm 3, the headline) and its deflated mixed form against VarCG (Algorithm 1, "
                    "64 sequential Lanczos steps), VarBL (Algorithm 2, 8 block steps of 64) and RIOT-PSAS "
                    "(Algorithm 4, 512 dual columns, FP64 dual products); cost reduction of Eq. 3 in FP64",
            "riot_mixed": {"ms_per_call": ms, "cost_reduction": red_mixed},
            **comparators}
    if deflated:
        line["deflated_mixed"] = deflated
    if fp64:
        line["fp64_gpu_form"] = fp64
    if bc:
        line["bc_transport"] = bc
    if batch:
        line["batch_windows"] = batch
    if learned:
        line["learned_sketch"] = learned
    if precond:
        line["precond_rotation"] = precond
    cs = clk.summary()
    if cs:
        line["clocks"] = cs
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import _clib
        _clib.build()
        cores = host_cores()
        try:
            d1, e1, r1 = cpu_oracle_rate(args.cpu_seconds / 2, 1)
            dn, en, rn = cpu_oracle_rate(args.cpu_seconds / 2, cores)
            line["cpu_baseline"] = {"value": rn, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": "%d Hessian-vector products of the same window in %.1f s on %d "
                                              "processes (FP64 C TL/AD + numpy L, one thread each, probes "
                                              "independent)" % (dn, en, cores),
                                    "one_core": {"value": r1, "products": d1, "seconds": e1}}
        except Exception as e:   # the headline line must not be lost to the CPU side
            line["cpu_baseline"] = {"error": str(e), "kind": "oracle", "cores": cores}
    if rank == 0:
        print(json.dumps(line))
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
