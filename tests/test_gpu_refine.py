"""GPU parity of mixed-precision refinement (cone_problem_set_inner: the
float32 problem is the instance, the CG steps apply a BF16 / FP8 copy of its
matrix) against the oracle's refinement mode, through the C ABI.

* iterates 1..20 (fixed 3 CG steps) within 1e-5 of the oracle's, and
  iterate 60 (after the exact refresh at 50) within 1e-4; the oracle's
  refined trajectory differs from its plain one, and from one without the
  refresh, by more than 3e-4, so the comparison sees which operand each pass
  applied;
* solves stop on, and return, the float32 problem's residuals: FP64
  rechecked residuals <= 1e-4 and objectives within 1e-4 of the oracle's
  optimum of the float32 instance;
* routing (the team engine refuses, auto picks the graph engine), argument
  errors, turning refinement off, the order of equilibration and set_inner,
  and serving == solo.
"""
import numpy as np
import pytest

from oracle import scs
from paper_1609_03488_b300 import synth
from tests.helpers import fp64_residuals, objective_rel_err, rel

pytestmark = pytest.mark.gpu
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


FAMILIES = {
    "lasso_bf16": (lambda: synth.lasso(m_d=301, p=151, seed=synth.BASE_SEED + 3), "bf16", None),
    "lasso_fp8": (lambda: synth.lasso(m_d=301, p=151, seed=synth.BASE_SEED + 3), "fp8", None),
    "lasso_fp8_equil": (lambda: synth.lasso(m_d=301, p=151, seed=synth.BASE_SEED + 3), "fp8", EQ),
    "lp_bf16": (lambda: synth.lp(m_d=301, n_x=151, density=0.05, seed=synth.BASE_SEED + 4), "bf16", None),
    "sparse_lasso_bf16": (lambda: synth.lasso_sparse(m_d=300, p=150, density=0.05, seed=35), "bf16", None),
}


def _refined(B, ctx, prob, storage, eq):
    P = B.cone_problem_create(ctx, prob)
    B.set_inner(P, synth.with_storage(prob["A"], storage))
    if eq:
        B.equilibrate(P, **eq)
    return P


@pytest.mark.parametrize("family", sorted(FAMILIES))
def test_refined_trajectory_matches_oracle(B, ctx, family):
    make, storage, eq = FAMILIES[family]
    prob = make()
    inner = synth.with_storage(prob["A"], storage)
    kw = dict(max_iters=60, check_interval=10 ** 6, linsys="cg", cg_fixed_steps=3, trajectory=60, equilibrate=eq)
    ref = scs.problem_solve(prob, inner=inner, **kw)
    plain = scs.problem_solve(prob, **kw)
    stale = scs.problem_solve(prob, inner=inner, refresh_interval=10 ** 9, **kw)
    assert rel(plain["traj_u"][19], ref["traj_u"][19]) > 3e-4
    assert rel(stale["traj_u"][59], ref["traj_u"][59]) > 3e-4
    P = _refined(B, ctx, prob, storage, eq)
    N = prob["A"]["n"] + prob["A"]["m"] + 1
    for k, tol in ((1, 1e-5), (5, 1e-5), (20, 1e-5), (60, 1e-4)):
        st = B.settings(max_iters=k, check_interval=10 ** 6, cg_fixed_iters=3)
        uv = np.empty(2 * N)
        info = B.cf_info()
        B.check(B.lib.solve(P.h, B.C.byref(st), None, None, None, None, B._ptr(uv), B.C.byref(info)), "solve")
        eu = rel(uv[:N], ref["traj_u"][k - 1])
        ev = rel(uv[N:], ref["traj_v"][k - 1])
        assert eu <= tol and ev <= tol, (family, k, eu, ev)


@pytest.mark.parametrize("family", ["lasso_bf16", "lasso_fp8", "lasso_fp8_equil", "lp_bf16"])
def test_refined_solutions_are_float32_optima(B, ctx, family):
    make, storage, eq = FAMILIES[family]
    prob = make()
    p_star = scs.problem_solve(prob, eps=1e-9, max_iters=400000)["pobj"]
    P = _refined(B, ctx, prob, storage, eq)
    info, x, y, s = B.solve(P, B.settings(eps=1e-5, max_iters=300000))
    assert info["status_name"] == "solved", info
    assert max(fp64_residuals(prob, x, y, s)) <= 1e-4, fp64_residuals(prob, x, y, s)
    assert objective_rel_err(prob["c"] @ x, p_star) <= 1e-4, (prob["c"] @ x, p_star)


def test_routing_and_arguments(B, ctx):
    prob = synth.lasso(m_d=200, p=100, seed=9)
    P = B.cone_problem_create(ctx, prob)
    assert B.team_info(P)[0]
    B.set_inner(P, synth.with_storage(prob["A"], "fp8"))
    ok, _, why = B.team_info(P)
    assert not ok and "inner operator" in why
    with pytest.raises(B.CfError) as e:
        B.solve(P, B.settings(max_iters=5, engine="team"))
    assert e.value.code == B.CF_E_INVALID
    info = B.solve(P, B.settings(eps=1e-4))[0]            # auto: graph engine
    assert info["status_name"] == "solved"
    wrong = synth.lasso(m_d=201, p=100, seed=9)
    with pytest.raises(B.CfError) as e:
        B.set_inner(P, wrong["A"])
    assert e.value.code == B.CF_E_INVALID
    other = B.Context(0)
    with pytest.raises(B.CfError) as e:
        B.set_inner(P, B.build_operator(other, prob["A"]))
    assert e.value.code == B.CF_E_INVALID
    # off again: the plain solve, bit for bit
    B.set_inner(P, None)
    assert B.team_info(P)[0]
    st = B.settings(eps=1e-5, engine="graph")
    a = B.solve(P, st)
    b = B.solve(B.cone_problem_create(ctx, prob), st)
    assert a[0]["iters"] == b[0]["iters"]
    np.testing.assert_array_equal(a[1], b[1])


def test_equilibration_order_does_not_matter(B, ctx):
    prob = synth.lasso(m_d=250, p=120, seed=10)
    inner = synth.with_storage(prob["A"], "fp8")
    P1 = B.cone_problem_create(ctx, prob)
    B.set_inner(P1, inner)
    B.equilibrate(P1, **EQ)
    P2 = B.cone_problem_create(ctx, prob)
    B.equilibrate(P2, **EQ)
    B.set_inner(P2, inner)
    st = B.settings(eps=1e-5)
    a, b = B.solve(P1, st), B.solve(P2, st)
    assert a[0]["status_name"] == "solved" and a[0]["iters"] == b[0]["iters"]
    for u, v in zip(a[1:], b[1:]):
        np.testing.assert_array_equal(u, v)


def test_refined_serving_equals_solo(B, ctx):
    probs = [synth.lasso(m_d=300, p=150, seed=2), synth.lp(m_d=200, n_x=100, density=0.05, seed=3),
             synth.lasso(m_d=260, p=130, seed=4)]
    Ps = [_refined(B, ctx, p, s, None) for p, s in zip(probs, ("fp8", "bf16", "bf16"))]
    st = B.settings(eps=1e-4)
    solo = [B.solve(P, st) for P in Ps]
    srv = B.Server(ctx, 100 << 20, 3)
    tickets = [(i, srv.submit(Ps[i], st)) for i in (0, 1, 2, 1)]
    for i, t in tickets:
        info, x, y, s = srv.wait(t, Ps[i])
        assert info["iters"] == solo[i][0]["iters"]
        np.testing.assert_array_equal(x, solo[i][1])
        np.testing.assert_array_equal(y, solo[i][2])
    srv.close()
