"""GPU parity of the lasso variants of Section 5.2 (sparse matrix and
convolution operators) and of the 2-D nonnegative deconvolution (the image
case of Section 2), against the FP64 oracle through the C ABI.

* sparse lasso (FP32 and BF16 values) on both engines: FP64-rechecked
  residuals <= 1e-4 and objective within 1e-4 of the oracle's optimum on the
  stored instance;
* convolution lasso, equilibrated (plain SCS crawls on the Gaussian blur), on
  both engines, against the oracle's equilibrated optimum;
* 2-D deconvolution on the graph engine (the team engine has no 2-D
  convolution leaf and says so): first 20 iterates within 1e-5 of the
  oracle's, solutions against scipy's NNLS, plain and equilibrated (the
  scalings then run as explicit elementwise stages).
"""
import numpy as np
import pytest
import scipy.optimize as so

from oracle import linop, scs
from paper_1609_03488_b300 import synth
from tests.helpers import fp64_residuals, objective_rel_err, rel

pytestmark = pytest.mark.gpu
ENGINES = ["graph", "team"]
EQ = dict(iters=10, probes=8, seed=0x5EED)


@pytest.fixture(scope="module")
def B():
    from paper_1609_03488_b300 import build
    build.build()
    from paper_1609_03488_b300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    return B.Context(0)


def _check(prob, info, x, y, s, p_star):
    assert info["status_name"] == "solved", info
    assert max(fp64_residuals(prob, x, y, s)) <= 1e-4, fp64_residuals(prob, x, y, s)
    assert objective_rel_err(prob["c"] @ x, p_star) <= 1e-4, (prob["c"] @ x, p_star)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_sparse_lasso(B, ctx, storage, engine):
    prob = synth.lasso_sparse(m_d=600, p=300, density=0.03, storage=storage, seed=31)
    ref = scs.problem_solve(prob, eps=1e-9, max_iters=200000)
    assert ref["status"] == scs.SOLVED
    P = B.cone_problem_create(ctx, prob)
    info, x, y, s = B.solve(P, B.settings(eps=1e-5, max_iters=200000, engine=engine))
    _check(prob, info, x, y, s, ref["pobj"])


@pytest.mark.parametrize("engine", ENGINES)
def test_convolution_lasso_equilibrated(B, ctx, engine):
    prob = synth.lasso_conv(p=300, L=60, seed=32)
    ref = scs.problem_solve(prob, eps=1e-8, max_iters=200000, equilibrate=EQ)
    assert ref["status"] == scs.SOLVED
    P = B.cone_problem_create(ctx, prob)
    B.equilibrate(P, **EQ)
    info, x, y, s = B.solve(P, B.settings(eps=1e-5, max_iters=300000, engine=engine))
    _check(prob, info, x, y, s, ref["pobj"])


def test_deconv2d_trajectory_matches_oracle(B, ctx):
    prob = synth.deconv2d(h=16, w=16, kh=5, kw=5, seed=33)
    ref = scs.problem_solve(prob, max_iters=20, check_interval=10 ** 6, linsys="cg", cg_fixed_steps=3,
                            trajectory=20)
    P = B.cone_problem_create(ctx, prob)
    ok, _, why = B.team_info(P)
    assert not ok and "2-D convolution" in why
    N = prob["A"]["n"] + prob["A"]["m"] + 1
    for k in (1, 5, 20):
        st = B.settings(max_iters=k, check_interval=10 ** 6, cg_fixed_iters=3)
        uv = np.empty(2 * N)
        info = B.cf_info()
        B.check(B.lib.solve(P.h, B.C.byref(st), None, None, None, None, B._ptr(uv), B.C.byref(info)), "solve")
        assert rel(uv[:N], ref["traj_u"][k - 1]) <= 1e-5 and rel(uv[N:], ref["traj_v"][k - 1]) <= 1e-5


@pytest.mark.parametrize("equilibrated", [False, True])
def test_deconv2d_solution(B, ctx, equilibrated):
    prob = synth.deconv2d(h=16, w=16, kh=5, kw=5, seed=34)
    K = linop.densify(prob["A"]["parts"][2]["parts"][0]["parts"][0])
    _, rnorm = so.nnls(K, prob["meta"]["b_obs"], maxiter=50000)
    P = B.cone_problem_create(ctx, prob)
    if equilibrated:
        B.equilibrate(P, **EQ)
    info, x, y, s = B.solve(P, B.settings(eps=1e-5, max_iters=300000))
    _check(prob, info, x, y, s, rnorm)
    with pytest.raises(B.CfError) as e:
        B.solve(P, B.settings(max_iters=5, engine="team"))
    assert e.value.code == B.CF_E_INVALID
