"""Pins of the oracle's mixed-precision refinement mode (``scs.solve(inner=)``,
the reading of Section 5.2's low-precision operands in which the float32
matrix stays the instance and BF16 / FP8 copies only drive the CG steps)
against facts outside it:

* with the exact operand as the inner one, the carried vectors equal the
  recomputed ones in exact arithmetic, so the iterates are the plain CG
  iteration's (a wrong sign or a dropped term in the carrying fails here);
* with BF16 / FP8 inner operands, the solutions satisfy the float32 lasso's
  own subgradient optimality conditions and reach HiGHS's optimum of the
  float32 LP, while the optimum of the quantised instance (the other reading)
  violates them by orders of magnitude more;
* a planted mistake (the exact refresh dropped) leaves the iteration on the
  wrong problem.
"""
import numpy as np
import pytest
import scipy.optimize as so

from oracle import linop, scs
from paper_1609_03488_b300 import synth
from tests.helpers import objective_rel_err, rel

EQ = dict(iters=10, probes=8, seed=0x5EED)


def _lasso_kkt_violation(prob, x):
    """Largest violation, relative to lam, of the lasso's subgradient
    conditions on the float32 matrix: |D^T (D x - b)|_i <= lam everywhere,
    = -lam sign(x_i) where x_i != 0."""
    D = prob["meta"]["D"].astype(np.float64)
    p, lam = prob["meta"]["p"], prob["meta"]["lam"]
    xx = x[:p]
    g = D.T @ (D @ xx - prob["meta"]["b_obs"])
    out = max(0.0, float(np.max(np.abs(g))) - lam) / lam
    nz = np.abs(xx) > 1e-7
    if nz.any():
        out = max(out, float(np.max(np.abs(g[nz] + lam * np.sign(xx[nz])))) / lam)
    return out


def test_exact_inner_operand_gives_the_plain_iteration():
    prob = synth.lasso(m_d=120, p=60, seed=41)
    kw = dict(max_iters=60, check_interval=10 ** 6, linsys="cg", cg_fixed_steps=3, trajectory=60)
    plain = scs.problem_solve(prob, **kw)
    ref = scs.problem_solve(prob, inner=prob["A"], refresh_interval=7, **kw)
    for k in (0, 6, 7, 30, 59):
        assert rel(ref["traj_u"][k], plain["traj_u"][k]) <= 1e-10
        assert rel(ref["traj_v"][k], plain["traj_v"][k]) <= 1e-10


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_refined_lasso_meets_the_float32_optimality_conditions(storage):
    prob = synth.lasso(m_d=200, p=100, seed=42)
    inner = synth.with_storage(prob["A"], storage)
    ref = scs.problem_solve(prob, eps=1e-7, max_iters=200000, linsys="cg", inner=inner)
    assert ref["status"] == scs.SOLVED
    assert _lasso_kkt_violation(prob, ref["x"]) <= 1e-5
    # the quantised instance's optimum is a different point
    quant = dict(prob, A=inner)
    other = scs.problem_solve(quant, eps=1e-9, max_iters=200000)
    assert other["status"] == scs.SOLVED
    assert _lasso_kkt_violation(prob, other["x"]) >= 2e-4


def test_refined_equilibrated_lasso_meets_the_float32_optimality_conditions():
    prob = synth.lasso(m_d=200, p=100, seed=43)
    ref = scs.problem_solve(prob, eps=1e-7, max_iters=200000, linsys="cg",
                            inner=synth.with_storage(prob["A"], "fp8"), equilibrate=EQ)
    assert ref["status"] == scs.SOLVED
    assert _lasso_kkt_violation(prob, ref["x"]) <= 1e-5


def test_refined_lp_reaches_the_float32_optimum():
    prob = synth.lp(m_d=60, n_x=30, density=0.2, seed=44)
    D = linop.densify(prob["A"]["parts"][0])
    hi = so.linprog(prob["c"], A_ub=D, b_ub=prob["b"][:60], bounds=(0, None), method="highs")
    ref = scs.problem_solve(prob, eps=1e-7, max_iters=100000, linsys="cg",
                            inner=synth.with_storage(prob["A"], "bf16"), equilibrate=EQ)
    assert ref["status"] == scs.SOLVED
    assert objective_rel_err(ref["pobj"], hi.fun) <= 1e-6
    pri, dual, gap = scs.residuals(scs.Operator(prob["A"]), prob["b"], prob["c"], ref["x"], ref["y"], ref["s"])
    assert max(pri, dual, gap) <= 1e-7


def test_planted_mistake_without_refresh_misses_the_optimum():
    """Dropping the exact refresh leaves A z_x and A^T A z_x on the FP8
    operand for good: the iteration then solves a mixture of the two
    problems and never meets the float32 conditions."""
    prob = synth.lasso(m_d=200, p=100, seed=42)
    bad = scs.problem_solve(prob, eps=1e-7, max_iters=5000, linsys="cg",
                            inner=synth.with_storage(prob["A"], "fp8"), refresh_interval=10 ** 9)
    assert bad["status"] != scs.SOLVED or _lasso_kkt_violation(prob, bad["x"]) > 1e-3


def test_refinement_arguments():
    prob = synth.lasso(m_d=40, p=20, seed=45)
    with pytest.raises(ValueError):
        scs.problem_solve(prob, inner=prob["A"])                      # needs the CG solver
    other = synth.lasso(m_d=41, p=20, seed=45)
    with pytest.raises(ValueError):
        scs.problem_solve(prob, linsys="cg", inner=other["A"])        # shape
