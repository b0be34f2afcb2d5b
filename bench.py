#!/usr/bin/env python
"""Benchmark of the SCS-style ADMM hot path.

Headline (the JSON line's ``value``): the large 1-D nonnegative
deconvolution (n = 1e6 signal, Gaussian kernel of length 1000, sigma = 100,
1% nonnegative support with Exp(1) values, noise 0.01; cone form with
n = 1,000,001 variables and m = 2,001,000 rows), equilibrated, FFT
convolution.  A step is one solve of that cone program from the standard
starting point, capped at --iters-per-step ADMM iterations (residual checks
every 10 iterations), with the problem resident in HBM; the metric is ADMM
iterations per second.

Beside it, on the same line: time to an accurate solution (residuals <= 1e-4
and objective within 1e-4 of the FP64 optimum, cold and warm, at the tuned
and the default CG prefactor), the dominant kernel's roofline against the
measured FMA rate, the per-iteration HBM fraction, the end-to-end rate from
host buffers, the oracle on the host cores, and the other half of the
metric: a batch of 512 sparse LPs (batched solves/s) and a Poisson serving
trace (solves/s, p50/p99).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--no-secondary]
"""
from __future__ import annotations

import os

# BLAS / OpenMP threads of the host-side oracle legs: every core this process
# may run on (set before numpy is imported).
AFFINITY_CORES = len(os.sched_getaffinity(0))
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, str(AFFINITY_CORES))

import argparse  # noqa: E402
import json  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

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
EQUIL = dict(iters=10, probes=8, seed=0x5EED)
# CG tolerance prefactor of the large deconvolution's headline solve,
# measured on this instance (time to 1e-4 with the FFT convolution at
# 1 / 3 / 10 / 30: 2.08 / 3.71 / 0.93 / 0.51 s); the library default is 1.
DECONV_CG_TOL_REL = 30.0
LIB_CG_TOL_REL = 1.0
# accuracy the time-to-solution legs ask for: FP64-accumulated residuals
# <= 1e-4 and the objective within 1e-4 of the FP64 optimum
ACCURACY = 1e-4
EPS_LADDER = (1e-4, 5e-5, 2e-5, 1e-5)
OPTIMUM_FILE = os.path.join(ROOT, "tests", "golden", "deconv_large_optimum.json")
# DRAM bytes (read + write) per launch from one ncu capture of each kernel on
# this workload, valid only for the kernel source they were taken on (source
# hash): the direct-sum convolution, and the scaled FFT convolution forward
# pass that the equilibrated solver runs.
CONV_NCU = {"traffic_bytes": 4029184, "src_sha256_16": "f372736cf1cfc748"}
FFT_NCU = {"traffic_bytes": 12080640, "src_sha256_16": "db62dd580fdc0efa"}
FFT_AUTO_LP = (256, 2048)   # padded tap counts for which the library's auto method takes the FFT
FFT_2048_MAX_LP = 1024      # the library takes 2048-point transforms up to this many padded taps when
                            # 4096-point ones would give fewer pairs than twice the SMs


def fft_size(Lp, n_out, sm_count):
    """The transform size the library picks for a convolution leaf."""
    v4096 = 4096 - Lp + 1
    pairs4096 = -(-n_out // (2 * v4096))
    return 2048 if (Lp <= FFT_2048_MAX_LP and pairs4096 < 2 * sm_count) else 4096
FP32_LANES_PER_SM = 128
L2_FLUSH_BYTES = 256 << 20
L2_BYTES = 126 << 20        # B300 L2: operands above this stream from HBM even back to back
PROFILE = False   # set by --profile


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--iters-per-step", type=int, default=400)
    ap.add_argument("--ttc-max-iters", type=int, default=20000,
                    help="iteration cap of the time-to-solution solves (0 = skip them)")
    ap.add_argument("--cpu-iters", type=int, default=6, help="ADMM iterations of the oracle sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the LP-batch and serving legs of the default run")
    ap.add_argument("--workload", default="deconv",
                    choices=["deconv", "deconv-small", "lasso", "lp-batch", "serve", "ops", "paper-lasso",
                             "paper-deconv"],
                    help="deconv (default): the large deconvolution (+ LP batch and serving legs); "
                         "lp-batch / serve: those legs alone")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--storage", default="bf16", choices=["fp32", "bf16", "fp8"], help="lasso: operand storage")
    ap.add_argument("--inner", default="none", choices=["none", "bf16", "fp8"],
                    help="lasso: mixed-precision refinement, the CG steps on a copy of D in this storage "
                         "(the instance stays --storage)")
    ap.add_argument("--single-sample", type=int, default=32,
                    help="lp-batch: LPs solved one at a time in FP32 for the single-solve comparison")
    ap.add_argument("--serve-seconds", type=float, default=20.0, help="serve: length of the arrival trace")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: mean arrival rate (req/s)")
    ap.add_argument("--pool", type=int, default=48, help="serve: distinct problem instances the requests draw from")
    ap.add_argument("--slots", type=int, default=32, help="serve: concurrent solves")
    ap.add_argument("--queue", type=int, default=64,
                    help="serve: outstanding requests beyond which arrivals are shed by the client")
    ap.add_argument("--sweep-seconds", type=float, default=4.0, help="serve: length of each sustainable-rate run")
    ap.add_argument("--budget-gb", type=float, default=60.0, help="serve: device memory budget")
    ap.add_argument("--lp-max-iters", type=int, default=50000)
    ap.add_argument("--engine", default="auto", choices=["auto", "graph", "team", "grid"],
                    help="solver program (auto: team engine for supported problems with small operator passes)")
    ap.add_argument("--tune-iters", type=int, default=20, help="lp-batch: ADMM iterations per autotuner candidate")
    ap.add_argument("--equil", default="on", choices=["on", "off"],
                    help="matrix-free equilibration of each problem (10 Ruiz steps x 8 probes)")
    ap.add_argument("--cg-tol-rel", type=float, default=None,
                    help="CG tolerance prefactor (default: 30 for the equilibrated large deconvolution, "
                         "else the library's 1)")
    ap.add_argument("--conv", default="auto", choices=["auto", "direct", "fft"],
                    help="deconv: how the 1-D convolution leaf is evaluated (auto: FFT for 256..2048 taps)")
    ap.add_argument("--profile", action="store_true",
                    help="bracket the measured region with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--reps", type=int, default=20, help="ops: timed launches per operator leaf")
    ap.add_argument("--host-loop", action="store_true",
                    help="launch the same kernels from the host instead of one CUDA graph per solve "
                         "(for profilers that cannot see kernels inside graph conditional nodes)")
    return ap.parse_args()


def conv_src_sha(fft=False):
    import hashlib
    if fft:
        src = "".join(open(os.path.join(ROOT, "paper_1609_03488_b300", "csrc", f)).read()
                      for f in ("k_fftconv.cu", "fftconv.cuh"))
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


def deconv_optimum():
    """The stored FP64 optimum t* of the large deconvolution (written by the
    oracle's exact NNLS; the value is a cone-program objective, not a kernel
    output), or None."""
    try:
        g = json.load(open(OPTIMUM_FILE))
    except Exception:
        return None
    if dict(g["instance"]) != dict(WORKLOAD):
        return None
    return {"t_star": 0.5 * (g["t_lo"] + g["t_hi"]), "bracket": [g["t_lo"], g["t_hi"]],
            "nnls_seconds_build_host": g.get("seconds"), "support": g.get("support_size")}


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



# ------------------------------------------------------------------ oracle legs
# The FP64 oracle is test infrastructure; bench.py runs it only here: the
# cpu_baseline legs and the --impl reference arm.
def cpu_sample(prob, iters, label, equilibrate=None, cg_tol_rel=1.0):
    """The FP64 oracle (matrix-free, CG linear solves) on the same instance
    and the same iteration as the GPU (equilibrated when the GPU is, same CG
    prefactor) for a bounded number of ADMM iterations on the host cores."""
    from oracle import equil as oequil, scs
    t0 = time.perf_counter()
    eq = None
    if equilibrate is not None:
        eq = oequil.equilibrate(scs.Operator(prob["A"]), prob["cone"], prob["b"], prob["c"], **equilibrate)
    t_eq = time.perf_counter() - t0
    r = scs.solve(prob["A"], prob["b"], prob["c"], prob["cone"], eps=1e-4, max_iters=iters, linsys="cg",
                  equil=eq, cg_tol_rel=cg_tol_rel)
    return {"value": r["iters"] / r["t_iter"], "unit": METRIC, "cores": AFFINITY_CORES, "kind": "oracle",
            "sample": (f"{r['iters']} ADMM iterations of the same {label} instance, "
                       f"{'equilibrated (' + str(equilibrate['iters']) + ' Ruiz steps x ' + str(equilibrate['probes']) + ' probes, ' + format(t_eq, '.1f') + ' s, excluded)' if eq else 'unequilibrated'}, "
                       f"CG prefactor {cg_tol_rel:g} (FP64, matrix-free numpy.convolve operators, CG subspace "
                       f"solves; setup {r['t_setup']:.1f} s excluded, iterations {r['t_iter']:.1f} s)"),
            "threads": {"blas_omp": AFFINITY_CORES,
                        "note": "numpy.convolve, the oracle's dominant cost, runs on one core"}}


def fft_nnls_baseline(opt):
    """The independent FP64 solver of the deconvolution (exact NNLS with FFT
    convolutions, oracle/nnls_conv.py) timed on the host cores on the same
    generator at n = 1e5 (a bounded sample) to its certified optimum; the
    n = 1e6 instance's own solve time is the stored figure."""
    from oracle import nnls_conv
    p = synth.deconv(n_x=100_000, L=1000, sigma=100.0, support=0.01, seed=synth.BASE_SEED + 2)
    t0 = time.perf_counter()
    _, info = nnls_conv.nnls_conv(p["meta"]["kernel"], p["meta"]["b_obs"], 100_000, workers=AFFINITY_CORES)
    el = time.perf_counter() - t0
    return {"kind": "independent FP64 solver (exact active-set NNLS, FFT convolutions)",
            "sample": "n=1e5, L=1000, sigma=100, 1% support (same generator), solved to its certified optimum",
            "seconds": el, "cores": AFFINITY_CORES, "certified_rel_gap": info["gap"] / info["f"],
            "full_size_seconds_stored": opt.get("nnls_seconds_build_host") if opt else None,
            "full_size_note": "n=1e6 solve time recorded when the stored optimum was written (8-core build host)"}


def run_reference(args, rank):
    """The oracle arm: the FP64 oracle on the headline workload (the same
    equilibrated iteration and CG prefactor as the GPU's), each step a
    2-iteration solve; the equilibration and the setup g = M^-1 h run once,
    outside the steps, as the GPU's resident problem has them."""
    if rank != 0:
        return
    from oracle import equil as oequil, scs
    prob = synth.deconv(**WORKLOAD)
    eq = oequil.equilibrate(scs.Operator(prob["A"]), prob["cone"], prob["b"], prob["c"], **EQUIL)
    kw = dict(eps=1e-4, linsys="cg", equil=eq, cg_tol_rel=DECONV_CG_TOL_REL)
    for _ in range(args.warmup):
        scs.solve(prob["A"], prob["b"], prob["c"], prob["cone"], max_iters=1, **kw)
    iters, t_it, t_all = 0, 0.0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = scs.solve(prob["A"], prob["b"], prob["c"], prob["cone"], max_iters=2, **kw)
        t_all += time.perf_counter() - t0
        iters += r["iters"]
        t_it += r["t_iter"]
    value = iters / t_it
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_NAME,
                                             "step": "oracle solve capped at 2 ADMM iterations of the equilibrated "
                                                     "problem, CG prefactor 30 (setup excluded from value)"},
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": AFFINITY_CORES, "kind": "oracle",
                             "sample": f"{iters} ADMM iterations over {args.steps} steps of the full instance"},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def pct(v, q):
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if len(v) else None


# ------------------------------------------------------------------ LP batch and serving legs
def _gen(spec):
    """One generated problem (run in a spawned worker process)."""
    kind, kw = spec
    return getattr(synth, kind)(**kw)


def generate(specs, workers=None):
    """Generate problems in parallel on the host cores (spawned processes:
    safe after CUDA has started in this one)."""
    import multiprocessing as mp
    workers = max(1, min(workers or AFFINITY_CORES, len(specs), 16))
    if workers == 1:
        return [_gen(s) for s in specs]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_gen, specs, chunksize=1)


def run_lp_batch(args, B, ctx, torch):
    """Batch of sparse LPs (min c^T x, D x <= b, x >= 0; m ~ U{200..20000}, n = m/2,
    density ~ U[0.5%, 2%]): the batched BF16 form (one solve_batch call, one
    persistent launch) against the batched FP32 form and the FP32 single-solve
    form (one LP at a time), all to 1e-4."""
    sizes = synth.lp_batch_sizes(count=args.batch_count)
    t0 = time.perf_counter()
    probs32 = generate([("lp", dict(m_d=m, n_x=n, density=d, seed=sd, storage="fp32")) for m, n, d, sd in sizes])
    t_gen = time.perf_counter() - t0
    # the BF16 instances share the generated arrays; the library rounds the values
    probs16 = [dict(p, A=synth.with_storage(p["A"], "bf16")) for p in probs32]
    nnz = sum(len(p["A"]["parts"][0]["col"]) for p in probs32)
    st = B.settings(eps=1e-4, max_iters=args.lp_max_iters, engine=args.engine,
                    **({"cg_tol_rel": args.cg_tol_rel} if args.cg_tol_rel is not None else {}))
    Ps = [B.cone_problem_create(ctx, p) for p in probs16]
    t_eq = 0.0
    if args.equil == "on":
        t0 = time.perf_counter()
        for P in Ps:
            B.equilibrate(P, **EQUIL)
        torch.cuda.synchronize()
        t_eq = time.perf_counter() - t0
    tune = None
    if args.engine != "graph" and args.tune_iters > 0:
        tune = B.solve_batch_tune(Ps, iters=args.tune_iters)     # schedule search (not timed below)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos, *_ = B.solve_batch(Ps, st)
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

    def status_counts(ii):
        out = {}
        for i in ii:
            out[i["status_name"]] = out.get(i["status_name"], 0) + 1
        return out

    solved = [i for i in infos if i["status_name"] == "solved"]
    worst = max((max(i["pri_res"], i["dual_res"], i["gap"]) for i in solved), default=None)
    for P in Ps:
        P.close()
    # the same batch with FP32 operands (same schedule)
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
    # plain FP32 single-solve form (one LP at a time, whole-GPU graph engine)
    # on an evenly spaced sample
    st_single = B.settings(eps=1e-4, max_iters=args.lp_max_iters, engine="graph")
    idx = list(range(0, len(sizes), max(1, len(sizes) // args.single_sample)))[:args.single_sample]
    t_single, single = 0.0, []
    for k in idx:
        P = B.cone_problem_create(ctx, probs32[k])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info, *_ = B.solve(P, st_single)
        t_single += time.perf_counter() - t0
        single.append(info)
        P.close()
    del probs32, probs16
    single_rate = len(idx) / t_single
    return {"metric": "batched solves/s", "value": len(infos) / t_batch, "unit": "solves/s",
            "workload": f"{len(infos)} sparse LPs, m~U{{200..20000}}, n=m/2, density~U[0.5%,2%], total nnz {nnz}",
            "engine": args.engine, "autotune": tune, "roofline": hbm,
            "equilibration": ({"per_problem": EQUIL, "seconds_total": t_eq} if args.equil == "on" else None),
            "batched_bf16": {"solves_per_s": len(infos) / t_batch, "wall_s": t_batch, "p50_ms": pct(lat, 50),
                             "p99_ms": pct(lat, 99), "status": status_counts(infos),
                             "iters_p50": pct([i["iters"] for i in infos], 50),
                             "iters_max": max(i["iters"] for i in infos),
                             "admm_iters_total": sum(i["iters"] for i in infos),
                             "max_residual_solved": worst,
                             "gpu_launches": sum(i["kernel_launches"] for i in infos)},
            "batched_fp32": {"solves_per_s": len(infos32) / t_batch32, "wall_s": t_batch32,
                             "status": status_counts(infos32),
                             "gpu_launches": sum(i["kernel_launches"] for i in infos32)},
            "single_fp32": {"solves_per_s": single_rate, "sample": len(idx), "wall_s": t_single, "engine": "graph",
                            "status": status_counts(single)},
            "batched_over_single": (len(infos) / t_batch) / single_rate,
            "residuals": "FP64-accumulated on the GPU, original (unequilibrated) problem",
            "csr_roofline": {st_: csr_roofline(B, ctx, torch, storage=st_) for st_ in ("fp32", "bf16")},
            "generation_s": t_gen}


def serve_pool_specs(count, rng):
    """The serving trace's distinct instances, a third of each family at the
    serving workload's sizes: deconvolutions (n log-uniform in [1e3, 1e6],
    L = n/1000 clipped to [16, 1000]), BF16 dense lassos (m_d log-uniform in
    [1e3, 2e4], p = m_d/2) and sparse LPs (m log-uniform in [1e3, 1e5],
    n = m/2, density 1%)."""
    specs = []
    for k in range(count):
        seed = synth.BASE_SEED + 500 + k
        if k % 3 == 0:
            n = int(10 ** rng.uniform(3, 6))
            specs.append(("deconv", dict(n_x=n, L=int(min(1000, max(16, n // 1000))), support=0.01, seed=seed)))
        elif k % 3 == 1:
            m = int(10 ** rng.uniform(3, np.log10(2e4)))
            specs.append(("lasso", dict(m_d=m, p=m // 2, storage="bf16", seed=seed)))
        else:
            m = int(10 ** rng.uniform(3, 5))
            specs.append(("lp", dict(m_d=m, n_x=m // 2, density=0.01, seed=seed)))
    return specs


def serve_run(B, srv, Ps, st, rate, seconds, queue_cap, rng):
    """One Poisson arrival trace of `seconds` at `rate` requests/s, each
    request a solve of a uniformly drawn pool instance from the standard
    start.  The client sheds an arrival when `queue_cap` requests are already
    outstanding (admitted or queued in the server).  Latency = the server's
    queue + setup + solve time of each completed request."""
    n_arr = int(rng.poisson(rate * seconds))
    t_arr = np.sort(rng.uniform(0.0, seconds, n_arr))
    pick = rng.integers(0, len(Ps), n_arr)
    outstanding = {}
    lat, status, done_info, shed = [], {}, [], 0
    t0 = time.perf_counter()

    def reap(block):
        for tk in list(outstanding):
            try:
                info, *_ = srv.wait(tk, Ps[outstanding[tk]], timeout_ns=-1 if block else 0)
            except B.CfError as e:
                if e.code == B.CF_E_TIMEOUT:
                    continue
                raise
            del outstanding[tk]
            lat.append(1e3 * (info["queue_ns"] + info["setup_ns"] + info["solve_ns"]) / 1e9)
            status[info["status_name"]] = status.get(info["status_name"], 0) + 1
            done_info.append(info)

    last_reap = 0.0
    for ta, k in zip(t_arr, pick):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        if time.perf_counter() - last_reap > 1e-3:
            reap(False)
            last_reap = time.perf_counter()
        if len(outstanding) >= queue_cap:
            shed += 1
            continue
        outstanding[srv.submit(Ps[k], st)] = int(k)
    t_trace = time.perf_counter() - t0
    reap(True)
    t_all = time.perf_counter() - t0
    return {"offered_rate": rate, "trace_s": seconds, "arrivals": int(n_arr), "shed": shed,
            "completed": len(lat), "solves_per_s": len(lat) / t_all, "wall_s": t_all, "trace_wall_s": t_trace,
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "status": status,
            "gpu_launches": sum(i["kernel_launches"] for i in done_info)}


def run_serve(args, B, ctx, torch):
    """Serving: a pool of instances of the three families at the serving
    workload's sizes, resident and equilibrated; a Poisson trace of
    --serve-seconds at --rate requests/s through serve_submit / serve_wait
    (continuous batching on the GPU, client-side shedding beyond --queue
    outstanding requests), then a sustainable-rate sweep at fractions of the
    achieved rate, then alone-vs-mix equality of a few results."""
    rng = np.random.default_rng(synth.BASE_SEED + 77)
    specs = serve_pool_specs(args.pool, rng)
    t0 = time.perf_counter()
    probs = generate(specs)
    t_gen = time.perf_counter() - t0
    st = B.settings(eps=1e-4, max_iters=args.lp_max_iters, engine=args.engine)
    Ps = [B.cone_problem_create(ctx, p) for p in probs]
    if args.equil == "on":
        for P in Ps:
            B.equilibrate(P, **EQUIL)
    sizes = {"deconv_n": [p["A"]["n"] for p in probs if p["family"] == "deconv"],
             "lasso_m": [p["meta"]["D"].shape[0] for p in probs if p["family"] == "lasso"],
             "lp_m": [p["meta"]["m_d"] for p in probs if p["family"] == "lp"]}
    del probs
    srv = B.Server(ctx, int(args.budget_gb * (1 << 30)), args.slots)
    torch.cuda.synchronize()
    main = serve_run(B, srv, Ps, st, args.rate, args.serve_seconds, args.queue, rng)
    cap = main["solves_per_s"]
    sweep = []
    if args.sweep_seconds > 0:
        for frac in (0.25, 0.5, 0.75, 1.0):
            sweep.append(serve_run(B, srv, Ps, st, max(frac * cap, 0.5), args.sweep_seconds, args.queue, rng))
    sustainable = max((r["offered_rate"] for r in sweep if r["shed"] == 0 and r["completed"] >= 0.9 * r["arrivals"]),
                      default=None)
    # the same requests alone (one solve at a time, outside the server) give
    # the same answers as in the mix
    same = True
    for k in range(min(6, len(Ps))):
        tk = srv.submit(Ps[k], st)
        info_m, x_m, *_ = srv.wait(tk, Ps[k])
        info_a, x_a, *_ = B.solve(Ps[k], st)
        same &= bool(np.array_equal(x_a, x_m)) and info_a["iters"] == info_m["iters"]
    srv.close()
    for P in Ps:
        P.close()
    return {"metric": "served solves/s", "value": main["solves_per_s"], "unit": "solves/s",
            "workload": (f"pool of {len(Ps)} instances (1/3 each): deconvolution n in [1e3,1e6], BF16 dense lasso "
                         f"m in [1e3,2e4], sparse LP m in [1e3,1e5] (1%); Poisson arrivals at {args.rate:g}/s for "
                         f"{args.serve_seconds:g} s, each a solve from the standard start to 1e-4"),
            "slots": args.slots, "client_queue_cap": args.queue, "budget_gb": args.budget_gb,
            "trace": main, "sustainable_sweep": sweep, "sustainable_rate": sustainable,
            "p50_ms": main["p50_ms"], "p99_ms": main["p99_ms"], "engine": args.engine,
            "equilibration": EQUIL if args.equil == "on" else None, "pool_sizes": sizes,
            "alone_equals_mix_bitwise": same, "generation_s": t_gen}


_FLUSH_BUF = {}


def _flush_buffers(torch):
    dev = torch.cuda.current_device()
    if dev not in _FLUSH_BUF:
        d = torch.device("cuda", dev)
        _FLUSH_BUF[dev] = (torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=d),
                           torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=d),
                           torch.empty((), dtype=torch.float32, device=d))
    return _FLUSH_BUF[dev]


def time_apply(op, x, y, torch, stream, adjoint, reps=20, ws=None):
    """Average device time of one cf_op_apply_async launch with a cold L2:
    before each timed launch a 256 MB write evicts L2 and a 256 MB read of a
    second buffer then evicts the written lines (so the timed launch pays no
    write-backs of the flush), and CUDA events on the launching stream
    bracket the launch alone.  The host enqueues the launch while the flush
    runs, so the bracket holds no host time.  With PROFILE set, the timed
    launches (and the flushes) are the profiler's region."""
    wbuf, rbuf, sink = _flush_buffers(torch)
    for _ in range(3):
        op.apply_async(x, y, adjoint=adjoint, workspace=ws, stream=stream.cuda_stream)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.synchronize()
    if PROFILE:
        torch.cuda.profiler.start()
    with torch.cuda.stream(stream):
        for a, b in evs:
            wbuf.fill_(1.0)
            torch.sum(rbuf, dim=0, out=sink)
            a.record(stream)
            op.apply_async(x, y, adjoint=adjoint, workspace=ws, stream=stream.cuda_stream)
            b.record(stream)
    torch.cuda.synchronize()
    if PROFILE:
        torch.cuda.profiler.stop()
    return float(np.mean([a.elapsed_time(b) for a, b in evs])) / 1e3


def time_apply_warm(op, x, y, torch, adjoint, reps=20, ws=None):
    """Average device time of one launch with L2 warm and no host gaps:
    `reps` back-to-back launches captured in one CUDA graph and replayed."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        op.apply_async(x, y, adjoint=adjoint, workspace=ws, stream=s.cuda_stream)
        g.capture_begin()
        for _ in range(reps):
            op.apply_async(x, y, adjoint=adjoint, workspace=ws, stream=s.cuda_stream)
        g.capture_end()
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    g.replay()
    b.record()
    torch.cuda.synchronize()
    del g
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


def dense_roofline(B, ctx, torch, storage, D=None, m=20000, n=10000, reps=20):
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
    t_n = time_apply(op, xin, yout, torch, stream, False, reps=reps)
    t_t = time_apply(op, yin, xout, torch, stream, True, ws=ws, reps=reps)
    w_n = time_apply_warm(op, xin, yout, torch, False, reps=reps)
    w_t = time_apply_warm(op, yin, xout, torch, True, ws=ws, reps=reps)
    mat = m * n * esz + (m * 4 if storage == "fp8" else 0)
    by = mat + 4 * (m + n)
    pk = hbm_peak()
    # an operand larger than L2 streams from HBM on every launch: the
    # back-to-back time is an HBM time; a smaller one is timed cold
    big = mat > L2_BYTES
    p_n, p_t = (w_n, w_t) if big else (t_n, t_t)
    return {"storage": storage, "shape": [m, n], "matrix_bytes": mat, "peak_GBs": pk,
            "timing": ("ms: " + ("launches replayed back to back from one CUDA graph (operand larger than the "
                                 "126 MB L2)" if big else "cold L2") +
                       "; ms_cold: 256 MB write + 256 MB read of another buffer before each launch, CUDA events "
                       "around the launch; ms_back_to_back: launches replayed from one CUDA graph"),
            "gemv_n": {"bound": "hbm", "ms": 1e3 * p_n, "achieved": by / p_n / 1e9, "unit": "GB/s",
                       "frac": by / p_n / 1e9 / pk, "ms_cold": 1e3 * t_n, "ms_back_to_back": 1e3 * w_n},
            "gemv_t": {"bound": "hbm", "ms": 1e3 * p_t, "achieved": by / p_t / 1e9, "unit": "GB/s",
                       "frac": by / p_t / 1e9 / pk, "ms_cold": 1e3 * t_t, "ms_back_to_back": 1e3 * w_t}}


def run_ops(args, B, ctx, torch):
    """Operator leaves alone at the benchmark sizes (for kernel profiling):
    CSR (the largest LP's), dense 20000 x 10000 in BF16 / FP8 / FP32, and the
    large deconvolution's FFT convolution with scalings folded in."""
    out = {"metric": "operator HBM roofline", "value": None, "unit": "GB/s"}
    out["csr"] = {st_: csr_roofline(B, ctx, torch, storage=st_, reps=args.reps) for st_ in ("fp32", "bf16")}
    D = (np.random.default_rng(3).standard_normal((20000, 10000)) / np.sqrt(20000)).astype(np.float32)
    out["dense"] = {st_: dense_roofline(B, ctx, torch, st_, D, reps=args.reps) for st_ in ("bf16", "fp8", "fp32")}
    del D
    W = WORKLOAD
    prob = synth.deconv(**W)
    P = B.cone_problem_create(ctx, prob)
    B.equilibrate(P, **EQUIL)
    out["conv1d_fft_scaled"] = deconv_roofline(B, ctx, torch, torch.cuda.current_stream(), prob, W, P, "auto",
                                               True, False, reps=args.reps)
    P.close()
    out["value"] = out["dense"]["bf16"]["gemv_n"]["achieved"]
    return out


def csr_roofline(B, ctx, torch, m=20000, n=10000, density=0.02, storage="fp32", reps=20):
    """The largest LP's CSR operator alone: y = D x and x = D^T y."""
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(5)
    rp, col, val = synth.random_csr(rng, m, n, density)
    op = B.cf_op_csr(ctx, m, n, rp, col, val, storage)
    dev = torch.device("cuda", torch.cuda.current_device())
    x, y = torch.rand(n, device=dev), torch.rand(m, device=dev)
    xo, yo = torch.empty(n, device=dev), torch.empty(m, device=dev)
    t_n = time_apply(op, x, yo, torch, stream, False, reps=reps)
    t_t = time_apply(op, y, xo, torch, stream, True, reps=reps)
    w_n = time_apply_warm(op, x, yo, torch, False, reps=reps)
    w_t = time_apply_warm(op, y, xo, torch, True, reps=reps)
    vsz = 4 if storage == "fp32" else 2
    nnz = len(col)
    by = nnz * (4 + vsz) + 4 * (m + 1) + 4 * (m + n)
    pk = hbm_peak()
    return {"nnz": nnz, "storage": storage,
            "timing": "ms: cold L2 (256 MB write + 256 MB read of another buffer before each launch), CUDA "
                      "events around the launch; ms_back_to_back: launches replayed from one CUDA graph (the "
                      "32 MB operand then stays in L2)",
            "spmv": {"ms": 1e3 * t_n, "GBs": by / t_n / 1e9, "frac": by / t_n / 1e9 / pk, "ms_back_to_back": 1e3 * w_n},
            "spmv_t": {"ms": 1e3 * t_t, "GBs": by / t_t / 1e9, "frac": by / t_t / 1e9 / pk,
                       "ms_back_to_back": 1e3 * w_t},
            "bytes_per_launch": by, "peak_GBs": pk}



# ------------------------------------------------------------------ large deconvolution legs
def deconv_roofline(B, ctx, torch, stream, prob, W, P, conv_method, eq, small, reps=20):
    """The dominant kernel, timed live on the stream it runs on: the 1-D
    convolution leaf with the problem's equilibration scalings folded in
    (diag(D) K diag(E) applied through the library, the form every solver
    pass runs), forward and adjoint, against the measured FP32 FMA rate."""
    dev = torch.device("cuda", torch.cuda.current_device())
    L, nx = W["L"], W["n_x"]
    conv = B.cf_op_conv1d(ctx, prob["meta"]["kernel"], nx, conv_method)
    op, variant = conv, "unscaled"
    if eq:
        D, E, _, _ = B.scaling(P)
        # the SOC tail rows (after n_x nonnegative rows and the SOC head) and
        # the signal's columns of the cone-form operator
        Dk = np.ascontiguousarray(D[nx + 1:nx + 1 + nx + L - 1])
        Ek = np.ascontiguousarray(E[:nx])
        op = B.operator_compose(ctx, "product", [B.cf_op_diag(ctx, nx + L - 1, Dk), conv, B.cf_op_diag(ctx, nx, Ek)])
        variant = "scaled (equilibration diagonals folded in)"
    xin = torch.rand(nx, device=dev)
    yin = torch.rand(nx + L - 1, device=dev)
    xout = torch.empty_like(xin)
    yout = torch.empty_like(yin)
    # a product needs scratch in general (none is touched when the scalings fold in)
    ws = torch.empty(max(op.workspace_bytes(False), op.workspace_bytes(True)) // 4 + 1, device=dev)
    t_fwd = time_apply(op, xin, yout, torch, stream, False, ws=ws, reps=reps)
    t_adj = time_apply(op, yin, xout, torch, stream, True, ws=ws, reps=reps)
    w_fwd = time_apply_warm(op, xin, yout, torch, False, ws=ws, reps=reps)
    w_adj = time_apply_warm(op, yin, xout, torch, True, ws=ws, reps=reps)
    direct_fwd = 2.0 * L * (nx + L - 1)
    direct_adj = 2.0 * L * nx
    Lp = (L + 15) // 16 * 16
    fft = conv_method == "fft" or (conv_method == "auto" and FFT_AUTO_LP[0] <= Lp <= FFT_AUTO_LP[1])
    fft_n = fft_size(Lp, nx + L - 1, ctx.sm_count) if fft else None
    if fft:
        # overlap-save: per pair of segments one complex N-point transform
        # each way (5 N log2 N flops, the usual count) and the spectrum product
        v = fft_n - Lp + 1
        per_pair = 2 * 5 * fft_n * np.log2(fft_n) + 6 * fft_n
        flops_fwd = per_pair * np.ceil((nx + L - 1) / (2 * v))
        flops_adj = per_pair * np.ceil(nx / (2 * v))
    else:
        flops_fwd, flops_adj = direct_fwd, direct_adj
    # the launch as the solver runs it: back to back from a CUDA graph, its
    # operands just written (L2-resident); the cold-L2 launch is reported too
    achieved = (flops_fwd + flops_adj) / (w_fwd + w_adj) / 1e12
    fp32 = ctx.fma_rate(False) / 1e12
    fp64 = ctx.fma_rate(True) / 1e12
    sm_max = peaks().get("sm_max_mhz", 2032.0)
    derived = ctx.sm_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    ncu = FFT_NCU if fft else CONV_NCU
    traffic = ncu["traffic_bytes"] if (conv_src_sha(fft) == ncu["src_sha256_16"] and not small and eq) else None
    # bytes each launch must move: input, output (read too when
    # accumulating: not here), and the two scaling vectors when scaled
    by_fwd = 4.0 * (nx + (nx + L - 1)) + (4.0 * (nx + nx + L - 1) if eq else 0.0)
    by_adj = by_fwd
    return {"bound": "alu", "kernel": ("k_conv1d_fft" if fft else "k_conv1d") + ("<1>" if eq else "<0>"),
            "variant": variant, "achieved": achieved, "peak": fp32, "unit": "TFLOP/s", "frac": achieved / fp32,
            "traffic": traffic,
            "traffic_unit": "bytes per forward launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "peak_source": ("measured: cf_measure_fma_rate, float32 FMA chains over a full-occupancy grid, this run "
                            "(of measured)"),
            "peak_derived": derived,
            "peak_derived_source": f"{ctx.sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {sm_max:.0f} MHz",
            "fp64_fma_TFLOPs_measured": fp64,
            "per_launch_ms": {"forward": 1e3 * w_fwd, "adjoint": 1e3 * w_adj},
            "per_launch_timing": ("per_launch_ms: 20 launches back to back from one CUDA graph, CUDA events "
                                  "around the replay on its stream (as the solver's graph runs them, operands "
                                  "L2-resident); per_launch_ms_cold: 256 MB write + 256 MB read of another buffer "
                                  "before each launch, CUDA events around the launch"),
            "per_launch_ms_cold": {"forward": 1e3 * t_fwd, "adjoint": 1e3 * t_adj},
            "achieved_cold": (flops_fwd + flops_adj) / (t_fwd + t_adj) / 1e12,
            "flops_per_launch": {"forward": flops_fwd, "adjoint": flops_adj},
            "flops_definition": (f"FFT method: pairs x (2 x 5 N log2 N + 6 N), N = {fft_n}" if fft
                                 else "direct sum: 2 L per output"),
            "algorithmic_bytes_per_launch": {"forward": by_fwd, "adjoint": by_adj},
            "hbm_frac_of_launch": (by_fwd + by_adj) / (w_fwd + w_adj) / 1e9 / hbm_peak(),
            "direct_sum_equivalent_TFLOPs": (direct_fwd + direct_adj) / (w_fwd + w_adj) / 1e12}


def per_iteration_hbm(n, m, iters, cg_total, seconds):
    """Vector traffic of one ADMM iteration, (6N + 7 n k + 6 n) x 4 bytes
    (N = n + m + 1, k CG steps per iteration): the floor the iteration's
    vector passes cannot go below, against its measured time."""
    k = cg_total / max(iters, 1)
    N = n + m + 1
    by = (6.0 * N + 7.0 * n * k + 6.0 * n) * 4.0
    per = seconds / max(iters, 1)
    return {"ms": 1e3 * per, "cg_per_iter": k, "bytes": by, "bytes_formula": "(6N + 7 n k + 6 n) x 4",
            "achieved_GBs": by / per / 1e9, "peak_GBs": hbm_peak(), "frac": by / per / 1e9 / hbm_peak()}


def time_to_accuracy(args, B, ctx, torch, stream, prob, P, opt, eq, pinned, cg_rel=DECONV_CG_TOL_REL):
    """Time to an accurate solution of the headline problem: the first eps of
    the ladder whose solve ends with residuals <= 1e-4 and the objective
    within 1e-4 of the FP64 optimum; at the tuned and at the library's
    default CG prefactor.  Warm: the problem resident with its setup cached
    (CUDA events).  Cold: operator and problem created from pinned host
    buffers, equilibration, setup and solve, results copied back (wall)."""
    t_star = opt["t_star"] if opt else None
    n, m = prob["A"]["n"], prob["A"]["m"]
    out = {"criterion": (f"GPU residuals (FP64-accumulated) <= {ACCURACY:g} and |c^T x - t*|/(1+|t*|) <= "
                         f"{ACCURACY:g}, t* = FP64 optimum (exact NNLS, certified bracket)"),
           "t_star": t_star, "t_star_bracket": opt["bracket"] if opt else None}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, pref in (("tuned", cg_rel), ("default", LIB_CG_TOL_REL)):
        ladder = []
        for eps in EPS_LADDER:
            st = B.settings(max_iters=args.ttc_max_iters, eps=eps, cg_tol_rel=pref, engine=args.engine)
            e0.record(stream)
            info, x, *_ = B.solve(P, st)
            e1.record(stream)
            torch.cuda.synchronize()
            pobj = float(prob["c"] @ x)
            err = abs(pobj - t_star) / (1 + abs(t_star)) if t_star is not None else None
            ok = (info["status_name"] == "solved" and max(info["pri_res"], info["dual_res"], info["gap"]) <= ACCURACY
                  and err is not None and err <= ACCURACY)
            row = {"eps": eps, "warm_s": e0.elapsed_time(e1) / 1e3, "iters": info["iters"],
                   "status": info["status_name"], "pri": info["pri_res"], "dual": info["dual_res"],
                   "gap": info["gap"], "objective": pobj, "objective_rel_err": err,
                   "cg_per_iter": info["cg_iters_total"] / max(info["iters"], 1), "meets": ok}
            ladder.append(row)
            if ok:
                # the same solve cold, through the C ABI from host buffers
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ops = B.build_operator(ctx, prob["A"])
                Pk = B.Problem(ctx, ops, pinned["b"], pinned["c"], prob["cone"])
                if eq:
                    B.equilibrate(Pk, **EQUIL)
                info_c = B.solve(Pk, st, x=pinned["x"], y=pinned["y"], s=pinned["s"])[0]
                torch.cuda.synchronize()
                row["cold_s"] = time.perf_counter() - t0
                row["cold_iters"] = info_c["iters"]
                row["cold_setup_ms"] = info_c["setup_ns"] / 1e6
                Pk.close()
                ops.close()
                break
        out[name] = {"cg_tol_rel": pref, "ladder": ladder,
                     "first_accurate": next((r for r in ladder if r["meets"]), None)}
    acc = out["tuned"]["first_accurate"]
    out["seconds_warm"] = acc["warm_s"] if acc else None
    out["seconds_cold"] = acc.get("cold_s") if acc else None
    out["eps_used"] = acc["eps"] if acc else None
    return out


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



# ------------------------------------------------------------------ replicas
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
    global PROFILE
    args = parse()
    PROFILE = args.profile and args.workload in ("ops",)
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
    cg_rel = args.cg_tol_rel if args.cg_tol_rel is not None else (
        DECONV_CG_TOL_REL if (eq and not small) else LIB_CG_TOL_REL)
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
        if args.profile:
            torch.cuda.profiler.start()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            info = step()
            ev[k][1].record(stream)
            iters += info["iters"]
            launches += info["kernel_launches"] + 1
            infos.append(info)
        barrier()
        if args.profile:
            torch.cuda.profiler.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    t_max, it_total = reduce_over_ranks(ms, iters, dist, dev)
    value = it_total / (t_max / 1e3)
    cg_total = sum(i["cg_iters_total"] for i in infos)
    per_iter = per_iteration_hbm(n, m, iters, cg_total, ms / 1e3)

    roofline = deconv_roofline(B, ctx, torch, stream, prob, W, P, args.conv, eq, small)
    team = all(i["kernel_launches"] == 1 for i in infos)
    if team:
        # the whole solve is one launch of the team kernel, which runs this
        # problem on one CTA (one SM): its convolution flops per launch
        # (forward + adjoint passes: rhs, CG steps, checks, refreshes) over
        # the launch time, against one SM's share of the measured FP32 rate
        fl = 0.0
        ffwd, fadj = roofline["flops_per_launch"]["forward"], roofline["flops_per_launch"]["adjoint"]
        for i in infos:
            passes_adj = i["iters"] + i["cg_iters_total"] + i["checks"] + i["iters"] // 50
            passes_fwd = i["cg_iters_total"] + i["checks"] + i["iters"] // 50
            fl += passes_fwd * ffwd + passes_adj * fadj
        t_launch = ms / 1e3
        sm_peak = roofline["peak"] / ctx.sm_count
        roofline = {"bound": "alu", "kernel": "k_team (one-CTA team)", "achieved": fl / t_launch / 1e12,
                    "peak": sm_peak, "unit": "TFLOP/s", "frac": fl / t_launch / 1e12 / sm_peak, "traffic": None,
                    "peak_source": "measured FP32 FMA rate / SM count (the problem's team is one SM) (of measured)",
                    "note": "latency-bound: every vector (12 KB) stays on chip and the iteration is a chain of "
                            "CTA barriers; the other SMs are free for other problems",
                    "launch_ms": 1e3 * t_launch / len(infos),
                    "flops_per_launch": fl / len(infos),
                    "conv_kernel_alone": roofline}

    # ---- end to end through the C ABI with host buffers
    pinned = {"b": torch.from_numpy(prob["b"]).pin_memory().numpy(),
              "c": torch.from_numpy(prob["c"]).pin_memory().numpy(),
              "x": torch.empty(n, dtype=torch.float64).pin_memory().numpy(),
              "y": torch.empty(m, dtype=torch.float64).pin_memory().numpy(),
              "s": torch.empty(m, dtype=torch.float64).pin_memory().numpy()}
    e2e = None
    if not args.no_e2e:
        e2e_iters, e2e_t = 0, 0.0
        for k in range(args.steps):
            flush.zero_()
            barrier()
            t0 = time.perf_counter()
            ops = B.build_operator(ctx, prob["A"])
            Pk = B.Problem(ctx, ops, pinned["b"], pinned["c"], prob["cone"])
            if eq:
                B.equilibrate(Pk, **EQUIL)
            info = B.solve(Pk, st, x=pinned["x"], y=pinned["y"], s=pinned["s"])[0]
            torch.cuda.synchronize()
            e2e_t += time.perf_counter() - t0
            e2e_iters += info["iters"]
            Pk.close()
            ops.close()
        L = W["L"]
        e2e = {"value": e2e_iters / e2e_t, "unit": "iters/s",
               "h2d_bytes_per_step": int(4 * L + 8 * m + 8 * n),
               "d2h_bytes_per_step": int(8 * (n + 2 * m)),
               "includes": "operator + problem creation from pinned host buffers, "
                           + ("equilibration, " if eq else "") + "setup (g = M^-1 h), solve, x/y/s copied to host"}

    # ---- time to an accurate solution (objective against the FP64 optimum)
    ttc = None
    opt = None if small else deconv_optimum()
    if args.ttc_max_iters > 0 and not small:
        ttc = time_to_accuracy(args, B, ctx, torch, stream, prob, P, opt, eq, pinned, cg_rel)
    elif args.ttc_max_iters > 0:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st2 = B.settings(max_iters=args.ttc_max_iters, eps=1e-4, engine=st.engine, cg_tol_rel=cg_rel)
        e0.record(stream)
        info = B.solve(P, st2, x=xo, y=yo, s=so)[0]
        e1.record(stream)
        torch.cuda.synchronize()
        ttc = {"seconds": e0.elapsed_time(e1) / 1e3, "iters": info["iters"], "status": info["status_name"],
               "pri": info["pri_res"], "dual": info["dual_res"], "gap": info["gap"]}

    # ---- the other half of the metric: batched and served solves
    secondary = None
    if world == 1 and not small and not args.no_secondary:
        P.close()
        del flush
        torch.cuda.empty_cache()
        secondary = {}
        for name, fn in (("lp_batch", run_lp_batch), ("serve", run_serve)):
            with ClockSampler(local) as clk2:
                secondary[name] = fn(args, B, ctx, torch)
            secondary[name]["clocks"] = clk2.summary()

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_sample(prob, max(args.cpu_iters, 20000) if small else args.cpu_iters,
                         "n=1000" if small else "n=1e6", equilibrate=EQUIL if eq else None, cg_tol_rel=cg_rel)
        if not small:
            cpu["independent_solver"] = fft_nnls_baseline(opt)

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
                "cg_per_iter": cg_total / max(iters, 1),
                "per_iteration_hbm": per_iter,
                "time_to_accuracy": ttc, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "secondary": secondary,
                "gpu_launches": launches, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
