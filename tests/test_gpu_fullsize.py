"""GPU checks at the full sizes of the benchmark workloads, where a dense
oracle is out of reach: the oracle runs matrix-free (FP64, numpy.convolve)
for a few iterations, and the returned points are re-checked in FP64.

* large deconvolution, n = 1e6, L = 1000: first 5 iterates vs the oracle
  (same fixed CG step count); after 400 iterations the GPU's residuals agree
  with an FP64 recomputation from the returned point; y in K*, s in K.
* the same problem exactly as the benchmark solves it (equilibrated, FFT
  convolution with the scalings folded in, the benchmark's CG prefactor):
  the first 20 iterates vs the equilibrated oracle; and the solve the
  benchmark's time-to-accuracy leg reports meets FP64-rechecked residuals
  <= 1e-4 and an objective within 1e-4 of the FP64 optimum (the stored exact
  NNLS optimum, certified by its duality bracket).
* dense lasso, D 20000 x 10000 in FP32 / BF16 / FP8: solved to 1e-4,
  residuals re-checked in FP64 on the stored (quantised) instance.
"""
import json
import os

import numpy as np
import pytest

from oracle import cones, scs
from paper_1609_03488_b300 import synth
from tests.helpers import objective_rel_err, rel

OPTIMUM = os.path.join(os.path.dirname(__file__), "golden", "deconv_large_optimum.json")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1609_03488_b300 import build
    build.build()
    from paper_1609_03488_b300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    return B.Context(0)


@pytest.fixture(scope="module")
def large_deconv():
    return synth.deconv(n_x=1_000_000, L=1000, sigma=100.0, support=0.01, seed=synth.BASE_SEED + 2)


def test_large_deconvolution_first_iterates(B, ctx, large_deconv):
    prob = large_deconv
    k = 5
    ref = scs.problem_solve(prob, max_iters=k, check_interval=10 ** 6, linsys="cg", cg_fixed_steps=3,
                            trajectory=k)
    P = B.cone_problem_create(ctx, prob)
    N = prob["A"]["n"] + prob["A"]["m"] + 1
    for it in (1, k):
        st = B.settings(max_iters=it, check_interval=10 ** 6, cg_fixed_iters=3)
        uv = np.empty(2 * N)
        info = B.cf_info()
        B.check(B.lib.solve(P.h, B.C.byref(st), None, None, None, None, B._ptr(uv), B.C.byref(info)), "solve")
        assert rel(uv[:N], ref["traj_u"][it - 1]) <= 1e-5
        assert rel(uv[N:], ref["traj_v"][it - 1]) <= 1e-5


def test_large_deconvolution_residuals_after_400_iterations(B, ctx, large_deconv):
    prob = large_deconv
    P = B.cone_problem_create(ctx, prob)
    info, x, y, s = B.solve(P, B.settings(max_iters=400, eps=1e-4))
    assert info["iters"] == 400 and info["status_name"] == "max_iters"
    pri, dual, gap = scs.residuals(scs.Operator(prob["A"]), prob["b"], prob["c"], x, y, s)
    np.testing.assert_allclose([pri, dual, gap], [info["pri_res"], info["dual_res"], info["gap"]], rtol=2e-2)
    assert cones.dist_to_cone(s, prob["cone"]) <= 1e-6 * (1 + np.linalg.norm(s))
    assert cones.dist_to_dual_cone(y, prob["cone"]) <= 1e-6 * (1 + np.linalg.norm(y))


@pytest.fixture(scope="module")
def large_equil_trajectory(large_deconv):
    import bench
    return scs.problem_solve(large_deconv, max_iters=20, check_interval=10 ** 6, linsys="cg", cg_fixed_steps=3,
                             trajectory=20, equilibrate=bench.EQUIL)


@pytest.mark.parametrize("engine", ["graph", "grid"])
def test_large_deconvolution_benchmarked_form_first_20_iterates(B, ctx, large_deconv, large_equil_trajectory,
                                                                engine):
    import bench
    prob = large_deconv
    ref = large_equil_trajectory
    P = B.cone_problem_create(ctx, prob)          # conv method "auto": the FFT path at 1008 padded taps
    B.equilibrate(P, **bench.EQUIL)
    N = prob["A"]["n"] + prob["A"]["m"] + 1
    for it in (1, 5, 20):
        st = B.settings(max_iters=it, check_interval=10 ** 6, cg_fixed_iters=3,
                        cg_tol_rel=bench.DECONV_CG_TOL_REL, engine=engine)
        uv = np.empty(2 * N)
        info = B.cf_info()
        B.check(B.lib.solve(P.h, B.C.byref(st), None, None, None, None, B._ptr(uv), B.C.byref(info)), "solve")
        eu, ev = rel(uv[:N], ref["traj_u"][it - 1]), rel(uv[N:], ref["traj_v"][it - 1])
        assert eu <= 1e-5 and ev <= 1e-5, (it, eu, ev)


@pytest.mark.skipif(not os.path.exists(OPTIMUM), reason="stored optimum not written")
@pytest.mark.parametrize("engine", ["graph", "grid"])
def test_large_deconvolution_benchmarked_solve_is_accurate(B, ctx, large_deconv, engine):
    """Every solve of the benchmark's eps ladder that the GPU reports as
    accurate (its own residuals <= 1e-4, objective within 1e-4 of t*) is
    accurate when re-checked in FP64; the strictest eps of the ladder is."""
    import bench
    prob = large_deconv
    g = json.load(open(OPTIMUM))
    assert g["instance"] == bench.WORKLOAD
    t_star = 0.5 * (g["t_lo"] + g["t_hi"])
    assert g["t_hi"] - g["t_lo"] <= 1e-9 * t_star
    P = B.cone_problem_create(ctx, prob)
    B.equilibrate(P, **bench.EQUIL)
    op = scs.Operator(prob["A"])
    seen = []
    for eps in bench.EPS_LADDER:
        st = B.settings(eps=eps, max_iters=20000, cg_tol_rel=bench.DECONV_CG_TOL_REL, engine=engine)
        info, x, y, s = B.solve(P, st)
        err = objective_rel_err(prob["c"] @ x, t_star)
        claimed = (info["status_name"] == "solved" and err <= 1e-4
                   and max(info["pri_res"], info["dual_res"], info["gap"]) <= 1e-4)
        seen.append((eps, info["status_name"], info["iters"], err))
        if claimed or eps == bench.EPS_LADDER[-1]:
            pri, dual, gap = scs.residuals(op, prob["b"], prob["c"], x, y, s)
            assert max(pri, dual, gap) <= 1e-4, (eps, pri, dual, gap, seen)
            assert err <= 1e-4, seen
            assert cones.dist_to_cone(s, prob["cone"]) <= 1e-5 * (1 + np.linalg.norm(s))
            assert cones.dist_to_dual_cone(y, prob["cone"]) <= 1e-5 * (1 + np.linalg.norm(y))
        if claimed:
            break
    assert any(e <= 1e-4 for *_, e in seen), seen


@pytest.mark.parametrize("storage", ["fp32", "bf16", "fp8"])
def test_dense_lasso_full_size(B, ctx, storage):
    prob = synth.lasso(m_d=20000, p=10000, storage=storage, seed=synth.BASE_SEED + 3)
    P = B.cone_problem_create(ctx, prob)
    info, x, y, s = B.solve(P, B.settings(eps=1e-4, max_iters=20000))
    assert info["status_name"] == "solved", info
    op = scs.Operator(prob["A"])          # matrix-free FP64 on the stored values
    pri, dual, gap = scs.residuals(op, prob["b"], prob["c"], x, y, s)
    assert max(pri, dual, gap) <= 1e-4, (pri, dual, gap)
    assert cones.dist_to_cone(s, prob["cone"]) <= 1e-5 * (1 + np.linalg.norm(s))
    assert cones.dist_to_dual_cone(y, prob["cone"]) <= 1e-5 * (1 + np.linalg.norm(y))
    # the cone objective is the lasso objective at the returned x (up to the
    # residual): (1/2)||D x - b||^2 + lam ||x||_1 <= w + lam 1^T t
    from oracle import quant
    Dq = quant.dense_values(prob["meta"]["D"], storage)
    p, lam = 10000, prob["meta"]["lam"]
    xx = x[:p]
    f = 0.5 * np.sum((Dq @ xx - prob["meta"]["b_obs"]) ** 2) + lam * np.abs(xx).sum()
    assert abs(f - info["pobj"]) <= 1e-3 * (1 + abs(f))
