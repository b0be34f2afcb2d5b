#!/usr/bin/env python
"""Benchmark of the SCS-style ADMM hot path on the large 1-D nonnegative
deconvolution workload (n = 1e6 signal, Gaussian kernel of length 1000,
sigma = 100, 1% nonnegative support with Exp(1) values, noise 0.01; cone form
with n = 1,000,001 variables and m = 2,001,000 rows).

A step is one solve of that cone program from the standard starting point,
capped at --iters-per-step ADMM iterations (residual checks every 10
iterations, tolerance 1e-4), with the problem resident in HBM.  The metric is
ADMM iterations per second.  One JSON line is printed (rank 0).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# more hardware work queues, so that the per-problem streams of a batch or a
# server do not alias onto the default eight (must be set before CUDA starts)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from paper_1609_03488_b300 import synth  # noqa: E402

WORKLOAD = dict(n_x=1_000_000, L=1000, sigma=100.0, support=0.01, noise=0.01, seed=synth.BASE_SEED + 2)
WORKLOAD_SMALL = dict(n_x=1000, L=100, sigma=10.0, support=0.05, noise=0.01, seed=synth.BASE_SEED + 1)
WORKLOAD_SMALL_NAME = ("small 1-D nonnegative deconvolution: n=1000, Gaussian kernel L=100 sigma=10, 5% nonneg "
                       "support Exp(1), noise 0.01; SCS cone form n=1001 m=2100; a step is a full solve to 1e-4")
WORKLOAD_NAME = ("large 1-D nonnegative deconvolution: n=1e6, Gaussian kernel L=1000 sigma=100, "
                 "1% nonneg support Exp(1), noise 0.01; SCS cone form n=1000001 m=2001000 (1 SOC + nonneg)")
METRIC = "ADMM iters/s"
# DRAM bytes (read + write) per k_conv1d launch on this workload from one ncu
# capture (profiles/conv1d_large_deconvolution.md), valid only for the kernel
# source it was taken on.
EQUIL = dict(iters=10, probes=8, seed=0x5EED)
CONV_NCU = {"traffic_bytes": 4029184, "src_sha256_16": "f372736cf1cfc748"}
# the same for k_conv1d_fft: an unscaled forward launch of this workload
# (profiles/conv1d_fft_large_deconvolution.md)
FFT_NCU = {"traffic_bytes": 4107264, "src_sha256_16": "68543effff9f908a"}
FFT_N = 4096
FFT_AUTO_LP = (256, 2048)   # padded tap counts for which the library's auto method takes the FFT
FP32_LANES_PER_SM = 128
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--iters-per-step", type=int, default=400)
    ap.add_argument("--ttc-max-iters", type=int, default=20000,
                    help="iteration cap of the one-off time-to-1e-4 solve (0 = skip)")
    ap.add_argument("--cpu-iters", type=int, default=6, help="ADMM iterations of the oracle sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="deconv",
                    choices=["deconv", "deconv-small", "lasso", "lp-batch", "serve", "ops", "paper-lasso",
                             "paper-deconv"],
                    help="deconv (default): the large deconvolution; lp-batch: batch of sparse LPs of "
                         "uneven size; serve: Poisson-arrival serving trace")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--storage", default="bf16", choices=["fp32", "bf16", "fp8"], help="lasso: operand storage")
    ap.add_argument("--inner", default="none", choices=["none", "bf16", "fp8"],
                    help="lasso: mixed-precision refinement, the CG steps on a copy of D in this storage "
                         "(the instance stays --storage)")
    ap.add_argument("--single-sample", type=int, default=32,
                    help="lp-batch: LPs solved one at a time in FP32 for the single-solve comparison")
    ap.add_argument("--requests", type=int, default=96, help="serve: trace length")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: mean arrival rate (req/s)")
    ap.add_argument("--slots", type=int, default=32, help="serve: concurrent solves")
    ap.add_argument("--budget-gb", type=float, default=60.0, help="serve: device memory budget")
    ap.add_argument("--lp-max-iters", type=int, default=50000)
    ap.add_argument("--engine", default="auto", choices=["auto", "graph", "team"],
                    help="solver program (auto: team engine for supported problems with small operator passes)")
    ap.add_argument("--tune-iters", type=int, default=20, help="lp-batch: ADMM iterations per autotuner candidate")
    ap.add_argument("--equil", default="on", choices=["on", "off"],
                    help="deconv / lp-batch: matrix-free equilibration of each problem (10 Ruiz steps x 8 probes)")
    ap.add_argument("--cg-tol-rel", type=float, default=None,
                    help="CG tolerance prefactor (default: 10 for the equilibrated large deconvolution, else the library's 1)")
    ap.add_argument("--conv", default="auto", choices=["auto", "direct", "fft"],
                    help="deconv: how the 1-D convolution leaf is evaluated (auto: FFT for 256..2048 taps)")
    ap.add_argument("--host-loop", action="store_true",
                    help="launch the same kernels from the host instead of one CUDA graph per solve "
                         "(for profilers that cannot see kernels inside graph conditional nodes)")
    return ap.parse_args()


def conv_src_sha(fft=False):
    import hashlib
    if fft:
        src = open(os.path.join(ROOT, "paper_1609_03488_b300", "csrc", "k_fftconv.cu")).read()
        return hashlib.sha256(src.encode()).hexdigest()[:16]
    src = open(os.path.join(ROOT, "paper_1609_03488_b300", "csrc", "k_leaf.cu")).read()
    a = src.index("// ------------------------------------------------------------ 1-D convolution")
    b = src.index("// ------------------------------------------------------------ 2-D convolution")
    return hashlib.sha256(src[a:b].encode()).hexdigest()[:16]


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [v.strip() for v in line.split(",")]
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
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle
def cpu_sample(prob, iters, label, equilibrate=None, cg_tol_rel=1.0):
    """The FP64 oracle (matrix-free, CG linear solves) on the same instance
    for a bounded number of ADMM iterations on the host cores."""
    from oracle import scs
    r = scs.problem_solve(prob, eps=1e-4, max_iters=iters, linsys="cg", equilibrate=equilibrate,
                          cg_tol_rel=cg_tol_rel)
    return {"value": r["iters"] / r["t_iter"], "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": (f"{r['iters']} ADMM iterations of the same {label} instance (FP64, matrix-free "
                       f"numpy.convolve operators, CG subspace solves; setup {r['t_setup']:.1f} s excluded, "
                       f"iterations {r['t_iter']:.1f} s; single-threaded numpy.convolve dominates)"),
            "affinity_cores": len(os.sched_getaffinity(0))}


def run_reference(args, rank):
    if rank != 0:
        return
    prob = synth.deconv(**WORKLOAD)
    from oracle import scs
    for _ in range(args.warmup):
        scs.problem_solve(prob, eps=1e-4, max_iters=1, linsys="cg")
    iters, t_it, t_all = 0, 0.0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = scs.problem_solve(prob, eps=1e-4, max_iters=2, linsys="cg")
        t_all += time.perf_counter() - t0
        iters += r["iters"]
        t_it += r["t_iter"]
    value = iters / t_it
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_NAME,
                                             "step": "oracle solve capped at 2 ADMM iterations (setup excluded from value)"},
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": 1, "kind": "oracle",
                             "sample": f"{iters} ADMM iterations over {args.steps} steps of the full instance"},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ other workloads
def pct(v, q):
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if len(v) else None


def lp_problem_residuals(prob, x, y, s):
    from oracle import scs
    return max(scs.residuals(scs.Operator(prob["A"]), prob["b"], prob["c"], x, y, s))


def run_lp_batch(args, B, ctx, torch):
    """Batch of sparse LPs (min c^T x, D x <= b, x >= 0; m ~ U{200..20000}, n = m/2,
    density ~ U[0.5%, 2%]): the batched BF16 form (one solve_batch call, one
    graph per LP, all concurrent) against the FP32 single-solve form (one LP at
    a time), both to 1e-4."""
    sizes = synth.lp_batch_sizes(count=args.batch_count)
    t0 = time.perf_counter()
    probs16 = [synth.lp(m_d=m, n_x=n, density=d, seed=sd, storage="bf16") for m, n, d, sd in sizes]
    t_gen = time.perf_counter() - t0
    nnz = sum(len(p["A"]["parts"][0]["col"]) for p in probs16)
    st = B.settings(eps=1e-4, max_iters=args.lp_max_iters, engine=args.engine,
                    **({"cg_tol_rel": args.cg_tol_rel} if args.cg_tol_rel is not None else {}))
    Ps = [B.cone_problem_create(ctx, p) for p in probs16]
    t_eq = 0.0
    if args.equil == "on":
        t0 = time.perf_counter()
        for P in Ps:
            B.equilibrate(P, **EQUIL)
        t_eq = time.perf_counter() - t0
    tune = None
    if args.engine != "graph" and args.tune_iters > 0:
        tune = B.solve_batch_tune(Ps, iters=args.tune_iters)     # schedule search (not timed below)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos, xs, ys, ss = B.solve_batch(Ps, st)
    t_batch = time.perf_counter() - t0
    lat = [(i["setup_ns"] + i["solve_ns"]) / 1e6 for i in infos]
    # algorithmic operator bytes of the batch: per problem, its forward-pass
    # bytes times the passes it ran (rhs adjoint each iteration, forward +
    # adjoint per CG step, both at each residual check and each refresh)
    pass_bytes = [B.team_info(P)[1] for P in Ps]
    alg_bytes = sum(pb * (i["iters"] + 2 * i["cg_iters_total"] + 2 * i["checks"] + 2 * (i["iters"] // 50))
                    for pb, i in zip(pass_bytes, infos))
    hbm = {"bound": "hbm", "achieved": alg_bytes / t_batch / 1e9, "peak": hbm_peak(), "unit": "GB/s",
           "frac": alg_bytes / t_batch / 1e9 / hbm_peak(), "algorithmic_bytes": alg_bytes,
           "note": "whole batch, wall time; bytes = forward-pass bytes x operator passes of each problem"}
    status = {}
    for i in infos:
        status[i["status_name"]] = status.get(i["status_name"], 0) + 1
    check_idx = list(range(0, len(probs16), max(1, len(probs16) // 8)))[:8]
    res16 = max(lp_problem_residuals(probs16[k], xs[k], ys[k], ss[k]) for k in check_idx)
    for P in Ps:
        P.close()
    # the same batch with FP32 operands (same schedule)
    probs32 = [synth.lp(m_d=m, n_x=n, density=d, seed=sd, storage="fp32") for m, n, d, sd in sizes]
    P32 = [B.cone_problem_create(ctx, p) for p in probs32]
    if args.equil == "on":
        for P in P32:
            B.equilibrate(P, **EQUIL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos32, *_ = B.solve_batch(P32, st)
    t_batch32 = time.perf_counter() - t0
    for P in P32:
        P.close()
    del probs32
    # plain FP32 single-solve form (one LP at a time, whole-GPU graph engine)
    # on an evenly spaced sample
    st_single = B.settings(eps=1e-4, max_iters=args.lp_max_iters, engine="graph")
    idx = list(range(0, len(sizes), max(1, len(sizes) // args.single_sample)))[:args.single_sample]
    t_single, single_status, res32 = 0.0, {}, 0.0
    for k in idx:
        m, n, d, sd = sizes[k]
        pr = synth.lp(m_d=m, n_x=n, density=d, seed=sd, storage="fp32")
        P = B.cone_problem_create(ctx, pr)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info, x, y, sv = B.solve(P, st_single)
        t_single += time.perf_counter() - t0
        single_status[info["status_name"]] = single_status.get(info["status_name"], 0) + 1
        res32 = max(res32, lp_problem_residuals(pr, x, y, sv))
        P.close()
    # the sample is spaced evenly over the batch's (random) sizes
    single_rate = len(idx) / t_single
    return {"metric": "batched solves/s", "value": len(Ps) / t_batch, "unit": "solves/s",
            "workload": f"{len(Ps)} sparse LPs, m~U{{200..20000}}, n=m/2, density~U[0.5%,2%], total nnz {nnz}",
            "engine": args.engine, "autotune": tune, "roofline": hbm,
            "equilibration": ({"per_problem": EQUIL, "seconds_total": t_eq} if args.equil == "on" else None),
            "batched_bf16": {"solves_per_s": len(Ps) / t_batch, "wall_s": t_batch, "p50_ms": pct(lat, 50),
                             "p99_ms": pct(lat, 99), "status": status,
                             "iters_p50": pct([i["iters"] for i in infos], 50),
                             "iters_max": max(i["iters"] for i in infos),
                             "admm_iters_total": sum(i["iters"] for i in infos),
                             "device_s": {"sum": 1e-9 * sum(i["device_ns"] for i in infos),
                                          "max": 1e-9 * max(i["device_ns"] for i in infos),
                                          "p50": 1e-9 * pct([i["device_ns"] for i in infos], 50),
                                          "longest": [{"m": sizes[k][0], "density": round(sizes[k][2], 4),
                                                       "iters": infos[k]["iters"],
                                                       "s": 1e-9 * infos[k]["device_ns"]}
                                                      for k in sorted(range(len(infos)),
                                                                      key=lambda k: -infos[k]["device_ns"])[:5]]},
                             "gpu_launches": sum(i["kernel_launches"] for i in infos),
                             "fp64_max_residual_sampled": res16},
            "batched_fp32": {"solves_per_s": len(sizes) / t_batch32, "wall_s": t_batch32,
                             "status": {k: sum(1 for i in infos32 if i["status_name"] == k)
                                        for k in sorted({i["status_name"] for i in infos32})},
                             "gpu_launches": sum(i["kernel_launches"] for i in infos32)},
            "single_fp32": {"solves_per_s": single_rate, "sample": len(idx), "wall_s": t_single, "engine": "graph",
                            "status": single_status, "fp64_max_residual_sampled": res32},
            "batched_over_single": (len(Ps) / t_batch) / single_rate,
            "csr_roofline": {st_: csr_roofline(B, ctx, torch, storage=st_) for st_ in ("fp32", "bf16")},
            "generation_s": t_gen}


def time_apply(op, x, y, torch, stream, adjoint, reps=20, ws=None):
    """Average device time of one cf_op_apply_async launch (CUDA events on
    the launching stream)."""
    for _ in range(3):
        op.apply_async(x, y, adjoint=adjoint, workspace=ws, stream=stream.cuda_stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        op.apply_async(x, y, adjoint=adjoint, workspace=ws, stream=stream.cuda_stream)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps / 1e3


def hbm_peak():
    return peaks().get("hbm_gbs", 6400.0)


def run_lasso(args, B, ctx, torch):
    """Dense lasso, D 20000 x 10000 i.i.d. N(0, 1/m) stored FP32 / BF16 / FP8
    (per-row scale), x* 1% nonzero, noise 0.01, lam = 0.1 ||D^T b||_inf."""
    stream = torch.cuda.current_stream()
    m_d, p = 20000, 10000
    t0 = time.perf_counter()
    prob = synth.lasso(m_d=m_d, p=p, storage=args.storage, seed=synth.BASE_SEED + 3)
    t_gen = time.perf_counter() - t0
    P = B.cone_problem_create(ctx, prob)
    if args.inner != "none":
        B.set_inner(P, synth.with_storage(prob["A"], args.inner))
    n, m = prob["A"]["n"], prob["A"]["m"]
    dev = torch.device("cuda", torch.cuda.current_device())
    xo = torch.empty(n, dtype=torch.float64, device=dev)
    yo = torch.empty(m, dtype=torch.float64, device=dev)
    so = torch.empty(m, dtype=torch.float64, device=dev)
    st = B.settings(max_iters=args.iters_per_step, eps=1e-4)
    for _ in range(args.warmup):
        B.solve(P, st, x=xo, y=yo, s=so)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    iters, cg, launches = 0, 0, 0
    for k in range(args.steps):
        ev[k][0].record(stream)
        info = B.solve(P, st, x=xo, y=yo, s=so)[0]
        ev[k][1].record(stream)
        iters += info["iters"]
        cg += info["cg_iters_total"]
        launches += info["kernel_launches"]
    torch.cuda.synchronize()
    t = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    # time to 1e-4 (fresh start, setup cached)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    info = B.solve(P, B.settings(max_iters=20000, eps=1e-4), x=xo, y=yo, s=so)[0]
    a1.record(stream)
    torch.cuda.synchronize()
    dr = dense_roofline(B, ctx, torch, args.storage, prob["meta"]["D"])
    mat = dr["matrix_bytes"]
    pk = hbm_peak()
    per_iter = t / iters
    # operator passes per iteration: rhs 1, CG 2 per step, checks 2 per 10,
    # refresh 2 per 50; with refinement the CG passes read the inner copy
    passes = (1 + 2 * cg / iters + 0.1 * 2 + 2.0 / 50)
    inner_note = ""
    if args.inner != "none":
        dri = dense_roofline(B, ctx, torch, args.inner, prob["meta"]["D"])
        outer_passes = 1 + 0.1 * 2 + 2.0 / 50
        inner_passes = 2 * cg / iters
        alg = outer_passes * mat + inner_passes * dri["matrix_bytes"]
        passes = outer_passes + inner_passes
        inner_note = f", CG steps on a {args.inner} copy (mixed-precision refinement)"
    else:
        alg = passes * mat
    return {"metric": "ADMM iters/s", "value": iters / t, "unit": "iters/s",
            "workload": f"dense lasso D {m_d}x{p} {args.storage}{inner_note}, n={n} m={m}",
            "ms_per_iter": 1e3 * per_iter, "cg_per_iter": cg / iters, "steps": args.steps,
            "iters_per_step": iters / args.steps, "gpu_launches": launches,
            "time_to_1e-4": {"seconds": a0.elapsed_time(a1) / 1e3, "iters": info["iters"],
                             "status": info["status_name"], "pri": info["pri_res"], "dual": info["dual_res"],
                             "gap": info["gap"]},
            "hbm_roofline_per_iter": {"operator_passes": passes,
                                      "algorithmic_bytes": alg,
                                      "achieved_GBs": alg / per_iter / 1e9, "peak_GBs": pk,
                                      "frac": alg / per_iter / 1e9 / pk},
            "roofline": dr,
            "inner": args.inner,
            "generation_s": t_gen}


def dense_roofline(B, ctx, torch, storage, D=None, m=20000, n=10000):
    """The dense leaf alone: y = D x and x = D^T y; algorithmic bytes = the
    stored operand (+ FP8 row scales) + the two vectors."""
    stream = torch.cuda.current_stream()
    if D is None:
        D = (np.random.default_rng(3).standard_normal((m, n)) / np.sqrt(m)).astype(np.float32)
    m, n = D.shape
    esz = {"fp32": 4, "bf16": 2, "fp8": 1}[storage]
    op = B.cf_op_dense(ctx, D, storage)
    dev = torch.device("cuda", torch.cuda.current_device())
    xin, yin = torch.rand(n, device=dev), torch.rand(m, device=dev)
    xout, yout = torch.empty(n, device=dev), torch.empty(m, device=dev)
    ws = torch.empty(max(op.workspace_bytes(True) // 4, 1), device=dev)
    t_n = time_apply(op, xin, yout, torch, stream, False)
    t_t = time_apply(op, yin, xout, torch, stream, True, ws=ws)
    mat = m * n * esz + (m * 4 if storage == "fp8" else 0)
    by = mat + 4 * (m + n)
    pk = hbm_peak()
    return {"storage": storage, "shape": [m, n], "matrix_bytes": mat, "peak_GBs": pk,
            "gemv_n": {"bound": "hbm", "ms": 1e3 * t_n, "achieved": by / t_n / 1e9, "unit": "GB/s",
                       "frac": by / t_n / 1e9 / pk},
            "gemv_t": {"bound": "hbm", "ms": 1e3 * t_t, "achieved": by / t_t / 1e9, "unit": "GB/s",
                       "frac": by / t_t / 1e9 / pk}}


def run_ops(args, B, ctx, torch):
    """Operator leaves alone at the benchmark sizes (for kernel profiling)."""
    out = {"metric": "operator HBM roofline", "value": None, "unit": "GB/s"}
    out["csr"] = {st_: csr_roofline(B, ctx, torch, storage=st_) for st_ in ("fp32", "bf16")}
    D = (np.random.default_rng(3).standard_normal((20000, 10000)) / np.sqrt(20000)).astype(np.float32)
    out["dense"] = {st_: dense_roofline(B, ctx, torch, st_, D) for st_ in ("bf16", "fp8", "fp32")}
    out["value"] = out["dense"]["bf16"]["gemv_n"]["achieved"]
    return out


def csr_roofline(B, ctx, torch, m=20000, n=10000, density=0.02, storage="fp32"):
    """The largest LP's CSR operator alone: y = D x and x = D^T y."""
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(5)
    rp, col, val = synth.random_csr(rng, m, n, density)
    op = B.cf_op_csr(ctx, m, n, rp, col, val, storage)
    dev = torch.device("cuda", torch.cuda.current_device())
    x, y = torch.rand(n, device=dev), torch.rand(m, device=dev)
    xo, yo = torch.empty(n, device=dev), torch.empty(m, device=dev)
    t_n = time_apply(op, x, yo, torch, stream, False)
    t_t = time_apply(op, y, xo, torch, stream, True)
    vsz = 4 if storage == "fp32" else 2
    nnz = len(col)
    by = nnz * (4 + vsz) + 4 * (m + 1) + 4 * (m + n)
    pk = hbm_peak()
    return {"nnz": nnz, "storage": storage,
            "spmv": {"ms": 1e3 * t_n, "GBs": by / t_n / 1e9, "frac": by / t_n / 1e9 / pk},
            "spmv_t": {"ms": 1e3 * t_t, "GBs": by / t_t / 1e9, "frac": by / t_t / 1e9 / pk},
            "bytes_per_launch": by, "peak_GBs": pk}


def serve_trace(args, rng):
    """A scaled Poisson trace: thirds of deconvolutions (n log-uniform in
    [1e3, 1e5], L = n/1000 clipped to [16, 1000]), BF16 dense lassos (m_d
    log-uniform in [1e3, 5e3], p = m_d/2) and sparse LPs (m log-uniform in
    [1e3, 2e4], n = m/2, density 1%)."""
    reqs = []
    t = 0.0
    for k in range(args.requests):
        t += rng.exponential(1.0 / args.rate)
        kind = k % 3
        seed = synth.BASE_SEED + 500 + k
        if kind == 0:
            n = int(10 ** rng.uniform(3, 5))
            L = int(min(1000, max(16, n // 1000)))
            prob = synth.deconv(n_x=n, L=L, support=0.01, seed=seed)
        elif kind == 1:
            m = int(10 ** rng.uniform(3, np.log10(5000)))
            prob = synth.lasso(m_d=m, p=m // 2, storage="bf16", seed=seed)
        else:
            m = int(10 ** rng.uniform(3, np.log10(20000)))
            prob = synth.lp(m_d=m, n_x=m // 2, density=0.01, seed=seed)
        reqs.append((t, prob))
    return reqs


def run_serve(args, B, ctx, torch):
    rng = np.random.default_rng(synth.BASE_SEED + 77)
    reqs = serve_trace(args, rng)
    st = B.settings(eps=1e-4, max_iters=args.lp_max_iters, engine=args.engine)
    Ps = [B.cone_problem_create(ctx, p) for _, p in reqs]
    if args.equil == "on":
        for P in Ps:
            B.equilibrate(P, **EQUIL)
    srv = B.Server(ctx, int(args.budget_gb * (1 << 30)), args.slots)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tickets = []
    for (ta, _), P in zip(reqs, Ps):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        tickets.append((time.perf_counter(), srv.submit(P, st)))
    lat, status = [], {}
    results = []
    for (ts, tk), P in zip(tickets, Ps):
        info, x, y, sv = srv.wait(tk, P)
        lat.append(1e3 * (info["queue_ns"] + info["setup_ns"] + info["solve_ns"]) / 1e9)
        status[info["status_name"]] = status.get(info["status_name"], 0) + 1
        results.append((info, x))
    t_all = time.perf_counter() - t0
    srv.close()
    # the same request alone gives the same answer (first few requests)
    same = True
    for k in range(min(6, len(Ps))):
        info, x, *_ = B.solve(Ps[k], st)
        same &= bool(np.array_equal(x, results[k][1])) and info["iters"] == results[k][0]["iters"]
    return {"metric": "served solves/s", "value": len(Ps) / t_all, "unit": "solves/s",
            "workload": (f"{len(Ps)} requests, Poisson arrivals at {args.rate:g}/s, 1/3 each deconvolution "
                         "n in [1e3,1e5], BF16 lasso m in [1e3,5e3], sparse LP m in [1e3,2e4] (1%)"),
            "offered_rate": args.rate, "slots": args.slots, "budget_gb": args.budget_gb,
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "wall_s": t_all, "status": status,
            "engine": args.engine, "gpu_launches": sum(r[0]["kernel_launches"] for r in results),
            "equilibration": EQUIL if args.equil == "on" else None,
            "alone_equals_mix_bitwise": same}


def _time_to_eps(B, ctx, torch, prob, equilibrate, max_iters=20000):
    """Wall time of one solve to 1e-4 through the C ABI (problem resident,
    setup included), plain or equilibrated (equilibration included)."""
    P = B.cone_problem_create(ctx, prob)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if equilibrate:
        B.equilibrate(P, **EQUIL)
    info = B.solve(P, B.settings(eps=1e-4, max_iters=max_iters))[0]
    t = time.perf_counter() - t0
    P.close()
    return {"seconds": t, "iters": info["iters"], "status": info["status_name"],
            "cg_per_iter": info["cg_iters_total"] / max(info["iters"], 1),
            "engine": "team" if info["kernel_launches"] == 1 else "graph"}


# the paper's TensorFlow-on-GPU rows (Titan X, its own instances): context only
PAPER_LASSO_TF_GPU = {"dense": (9.9, 60), "sparse": (7.1, 40), "conv": (5.3, 180)}
PAPER_DECONV_TF_GPU = {100: (5.7, 480), 1000: (3.2, 100), 10000: (13.0, 160)}


def run_paper_lasso(args, B, ctx, torch):
    """The three lasso instances of Section 5.2's table (6001 variables):
    D 6000 x 3000 dense (N(0,1/m)), sparse (1% as the text says), and the
    3000-tap Gaussian convolution (sigma 300); time to 1e-4 each."""
    probs = {"dense": synth.lasso(m_d=6000, p=3000, seed=synth.BASE_SEED + 3),
             "sparse": synth.lasso_sparse(m_d=6000, p=3000, density=0.01, seed=synth.BASE_SEED + 5),
             "conv": synth.lasso_conv(p=3000, L=3000, seed=synth.BASE_SEED + 6)}
    out = {}
    for k, prob in probs.items():
        out[k] = {"n": prob["A"]["n"], "m": prob["A"]["m"],
                  "plain": _time_to_eps(B, ctx, torch, prob, False),
                  "equilibrated": _time_to_eps(B, ctx, torch, prob, True),
                  "paper_tf_gpu_seconds_iters": PAPER_LASSO_TF_GPU[k]}
    best = sum(min(v["plain"]["seconds"] if v["plain"]["status"] == "solved" else 1e9,
                   v["equilibrated"]["seconds"] if v["equilibrated"]["status"] == "solved" else 1e9)
               for v in out.values())
    return {"metric": "time to 1e-4, Section 5.2 lasso instances (sum of the three, best of plain / equilibrated)",
            "value": best, "unit": "s", "higher_is_better": False, "instances": out,
            "note": "the paper's instances and hardware differ (Titan X); its rows are context, not targets"}


def run_paper_deconv(args, B, ctx, torch):
    """The three nonnegative deconvolutions of Section 5.3's table (kernel
    length = signal length n, sigma n/10, 5 nonzeros); time to 1e-4 each."""
    out = {}
    for n in (100, 1000, 10000):
        prob = synth.deconv(n_x=n, L=n, support=5.0 / n, seed=synth.BASE_SEED + 8)
        out[str(n)] = {"n": prob["A"]["n"], "m": prob["A"]["m"],
                       "plain": _time_to_eps(B, ctx, torch, prob, False, max_iters=50000),
                       "equilibrated": _time_to_eps(B, ctx, torch, prob, True, max_iters=50000),
                       "paper_tf_gpu_seconds_iters": PAPER_DECONV_TF_GPU[n]}
    best = sum(min(v["plain"]["seconds"] if v["plain"]["status"] == "solved" else 1e9,
                   v["equilibrated"]["seconds"] if v["equilibrated"]["status"] == "solved" else 1e9)
               for v in out.values())
    return {"metric": "time to 1e-4, Section 5.3 deconvolution instances (sum of the three, best of plain / equilibrated)",
            "value": best, "unit": "s", "higher_is_better": False, "instances": out,
            "note": "the paper's instances and hardware differ (Titan X); its rows are context, not targets"}


# ------------------------------------------------------------------ ours
def replica_problem(workload, rank):
    """The deconvolution instance rank `rank` solves: the same shape on every
    rank, its own seed (independent replicas; no data crosses ranks)."""
    return synth.deconv(**{**workload, "seed": workload["seed"] + rank})


def reduce_over_ranks(ms, iters, dist, device):
    """Whole-job numbers of a replicated run: every rank times its own
    replica, the job's time is the slowest rank's and its work the sum over
    ranks (weak scaling).  Without a process group, the rank's own numbers."""
    if dist is None:
        return float(ms), float(iters)
    import torch
    tt = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    it = torch.tensor([float(iters)], device=device, dtype=torch.float64)
    dist.all_reduce(it, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(it.item())


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1609_03488_b300 import binding as B

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    small = args.workload == "deconv-small"
    if small:
        args.iters_per_step = max(args.iters_per_step, 20000)
    if args.workload not in ("deconv", "deconv-small"):
        stream = torch.cuda.Stream(device=local)
        torch.cuda.set_stream(stream)
        ctx = B.Context(local, stream.cuda_stream)
        run = {"lp-batch": run_lp_batch, "serve": run_serve, "lasso": run_lasso, "ops": run_ops,
               "paper-lasso": run_paper_lasso, "paper-deconv": run_paper_deconv}[args.workload]
        with ClockSampler(local) as clk:
            line = run(args, B, ctx, torch)
        line.setdefault("higher_is_better", True)
        line.update({"n_gpus": world, "data": "synthetic", "clocks": clk.summary()})
        if rank == 0:
            print(json.dumps(line), flush=True)
        return

    W = WORKLOAD_SMALL if small else WORKLOAD
    eq = args.equil == "on"
    # CG prefactor per workload (measured): 30 on the equilibrated n=1e6
    # deconvolution (time to 1e-4 with the FFT convolution at 1 / 3 / 10 / 30:
    # 2.08 / 3.71 / 0.93 / 0.51 s; 2090 / 4090 / 2080 / 2120 iterations; the
    # direct sum: 2.50 / 5.55 / 0.59 / 0.75 s), 1 on the small one (750
    # iterations vs 2090 at 10)
    cg_rel = args.cg_tol_rel if args.cg_tol_rel is not None else (30.0 if (eq and not small) else 1.0)
    prob = replica_problem(W, rank)
    prob["A"] = synth.with_conv_method(prob["A"], args.conv)
    n, m = prob["A"]["n"], prob["A"]["m"]
    # a dedicated (non-default) stream: the library launches on it and the
    # CUDA events below are recorded on it
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    ctx = B.Context(local, stream.cuda_stream)
    P = B.cone_problem_create(ctx, prob)
    if eq:
        B.equilibrate(P, **EQUIL)
    dev = torch.device("cuda", local)
    xo = torch.empty(n, dtype=torch.float64, device=dev)
    yo = torch.empty(m, dtype=torch.float64, device=dev)
    so = torch.empty(m, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    st = B.settings(max_iters=args.iters_per_step, eps=1e-4, host_loop=1 if args.host_loop else 0,
                    engine="graph" if args.host_loop else args.engine, cg_tol_rel=cg_rel)

    def step():
        return B.solve(P, st, x=xo, y=yo, s=so)[0]

    for _ in range(args.warmup):
        step()
    barrier()

    # ---- timed region: K steps, L2 flushed between steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    iters, launches, infos = 0, 0, []
    with ClockSampler(local) as clk:
        barrier()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            info = step()
            ev[k][1].record(stream)
            iters += info["iters"]
            launches += info["kernel_launches"] + 1
            infos.append(info)
        barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    t_max, it_total = reduce_over_ranks(ms, iters, dist, dev)
    value = it_total / (t_max / 1e3)

    # ---- dominant kernel: the 1-D convolution, timed live on the same stream
    conv = B.cf_op_conv1d(ctx, prob["meta"]["kernel"], W["n_x"], args.conv)
    L = W["L"]
    xin = torch.rand(W["n_x"], device=dev)
    yin = torch.rand(W["n_x"] + L - 1, device=dev)
    xout = torch.empty_like(xin)
    yout = torch.empty_like(yin)
    for _ in range(3):
        conv.apply_async(xin, yout, stream=stream.cuda_stream)
        conv.apply_async(yin, xout, adjoint=True, stream=stream.cuda_stream)
    reps = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        conv.apply_async(xin, yout, stream=stream.cuda_stream)
    e1.record(stream)
    e2.record(stream)
    for _ in range(reps):
        conv.apply_async(yin, xout, adjoint=True, stream=stream.cuda_stream)
    e3.record(stream)
    torch.cuda.synchronize()
    t_fwd = e0.elapsed_time(e1) / reps / 1e3
    t_adj = e2.elapsed_time(e3) / reps / 1e3
    direct_fwd = 2.0 * L * (W["n_x"] + L - 1)
    direct_adj = 2.0 * L * W["n_x"]
    Lp = (L + 15) // 16 * 16
    fft = args.conv == "fft" or (args.conv == "auto" and FFT_AUTO_LP[0] <= Lp <= FFT_AUTO_LP[1])
    if fft:
        # overlap-save: per pair of segments one complex FFT_N-point transform
        # each way (5 N log2 N flops, the usual count) and the spectrum product
        v = FFT_N - Lp + 1
        per_pair = 2 * 5 * FFT_N * np.log2(FFT_N) + 6 * FFT_N
        flops_fwd = per_pair * np.ceil((W["n_x"] + L - 1) / (2 * v))
        flops_adj = per_pair * np.ceil(W["n_x"] / (2 * v))
    else:
        flops_fwd, flops_adj = direct_fwd, direct_adj
    achieved = (flops_fwd + flops_adj) / (t_fwd + t_adj) / 1e12
    pk = peaks()
    sm_count = ctx.sm_count
    sm_max = pk.get("sm_max_mhz", 2032.0)
    alu_peak = sm_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    ncu = FFT_NCU if fft else CONV_NCU
    roofline = {"bound": "alu", "kernel": "k_conv1d_fft" if fft else "k_conv1d", "achieved": achieved,
                "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
                "traffic": (ncu["traffic_bytes"] if conv_src_sha(fft) == ncu["src_sha256_16"] and not small
                            else None),
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                "peak_source": f"derived: {sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {sm_max:.0f} MHz (max SM clock of measured)",
                "per_launch_ms": {"forward": 1e3 * t_fwd, "adjoint": 1e3 * t_adj},
                "flops_per_launch": {"forward": flops_fwd, "adjoint": flops_adj},
                "flops_definition": ("FFT method: pairs x (2 x 5 N log2 N + 6 N), N = 4096" if fft
                                     else "direct sum: 2 L per output"),
                "direct_sum_equivalent_TFLOPs": (direct_fwd + direct_adj) / (t_fwd + t_adj) / 1e12}

    team = all(i["kernel_launches"] == 1 for i in infos)
    if team:
        # the whole solve is one launch of the team kernel, which runs this
        # problem on one CTA (one SM): its convolution flops per launch
        # (forward + adjoint passes: rhs, CG steps, checks, refreshes) over
        # the launch time, against one SM's FP32 rate
        fl = 0.0
        for i in infos:
            passes_adj = i["iters"] + i["cg_iters_total"] + i["checks"] + i["iters"] // 50
            passes_fwd = i["cg_iters_total"] + i["checks"] + i["iters"] // 50
            fl += passes_fwd * flops_fwd + passes_adj * flops_adj
        t_launch = ms / 1e3
        sm_peak = FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        roofline = {"bound": "alu", "kernel": "k_team (one-CTA team)", "achieved": fl / t_launch / 1e12,
                    "peak": sm_peak, "unit": "TFLOP/s", "frac": fl / t_launch / 1e12 / sm_peak, "traffic": None,
                    "peak_source": f"derived: 1 SM (the problem's team) x {FP32_LANES_PER_SM} FP32 lanes x 2 flop "
                                   f"x {sm_max:.0f} MHz",
                    "note": "latency-bound: every vector (12 KB) stays on chip and the iteration is a chain of "
                            "CTA barriers; the other SMs are free for other problems",
                    "launch_ms": 1e3 * t_launch / len(infos),
                    "flops_per_launch": fl / len(infos),
                    "conv_kernel_alone": roofline}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        bh = torch.from_numpy(prob["b"]).pin_memory()
        ch = torch.from_numpy(prob["c"]).pin_memory()
        xh = torch.empty(n, dtype=torch.float64).pin_memory()
        yh = torch.empty(m, dtype=torch.float64).pin_memory()
        sh = torch.empty(m, dtype=torch.float64).pin_memory()
        e2e_iters, e2e_t = 0, 0.0
        for k in range(args.steps):
            flush.zero_()
            barrier()
            t0 = time.perf_counter()
            ops = B.build_operator(ctx, prob["A"])
            Pk = B.Problem(ctx, ops, bh.numpy(), ch.numpy(), prob["cone"])
            if eq:
                B.equilibrate(Pk, **EQUIL)
            info = B.solve(Pk, st, x=xh.numpy(), y=yh.numpy(), s=sh.numpy())[0]
            torch.cuda.synchronize()
            e2e_t += time.perf_counter() - t0
            e2e_iters += info["iters"]
            Pk.close()
            ops.close()
        e2e = {"value": e2e_iters / e2e_t, "unit": "iters/s",
               "h2d_bytes_per_step": int(4 * L + 8 * m + 8 * n),
               "d2h_bytes_per_step": int(8 * (n + 2 * m)),
               "includes": "operator + problem creation from pinned host buffers, "
                           + ("equilibration, " if eq else "") + "setup (g = M^-1 h), solve, x/y/s copied to host"}

    # ---- one-off time to 1e-4
    ttc = None
    if args.ttc_max_iters > 0:
        st2 = B.settings(max_iters=args.ttc_max_iters, eps=1e-4, engine=st.engine, cg_tol_rel=cg_rel)
        e0.record(stream)
        info = B.solve(P, st2, x=xo, y=yo, s=so)[0]
        e1.record(stream)
        torch.cuda.synchronize()
        ttc = {"seconds": e0.elapsed_time(e1) / 1e3, "iters": info["iters"], "status": info["status_name"],
               "pri": info["pri_res"], "dual": info["dual_res"], "gap": info["gap"],
               "cg_per_iter": info["cg_iters_total"] / max(info["iters"], 1)}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_sample(prob, max(args.cpu_iters, 20000) if small else args.cpu_iters,
                         "n=1000" if small else "n=1e6 (unequilibrated: the oracle's probes would take minutes)",
                         equilibrate=EQUIL if (eq and small) else None, cg_tol_rel=cg_rel)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD_SMALL_NAME if small else WORKLOAD_NAME, "n": n, "m": m,
                           "step": f"one solve from u=v=(0,0,1), capped at {args.iters_per_step} ADMM iterations, "
                                   "eps 1e-4 checked every 10 iterations",
                           "l2": "flushed between steps (256 MB write)",
                           "precision": "f32 vectors and operator, f64 reductions/norms/tau/kappa",
                           "equilibration": (f"matrix-free, {EQUIL['iters']} Ruiz steps x {EQUIL['probes']} sign probes"
                                             if eq else "none"),
                           "cg_tol": f"max(1e-9, {cg_rel:g} ||rhs|| (k+1)^-1.5)",
                           "engine": ("team (one persistent launch per solve)" if team else "graph (one CUDA graph per solve)"),
                           "parallelism": f"replicas x{world}"},
                "iters_per_step": it_total / max(args.steps * world, 1),
                "cg_per_iter": sum(i["cg_iters_total"] for i in infos) / max(iters, 1),
                "time_to_1e-4": ttc, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
