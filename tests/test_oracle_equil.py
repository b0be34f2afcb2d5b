"""Pins of the oracle's matrix-free equilibration (oracle/equil.py) against
facts outside it: the published SplitMix64 output sequence, the unbiasedness
of the random-sign row-norm estimator (checked against norms taken from the
explicit matrix), the balancing it produces, the cone rule (one factor per
second-order cone), and the invariance of the solution: the equilibrated
solve returns an optimum of the original problem (checked against HiGHS and
the unequilibrated solve), certificates included."""
import numpy as np
import pytest
import scipy.optimize as so

from oracle import cones, equil, linop, scs
from paper_1609_03488_b300 import synth
from tests.helpers import objective_rel_err


def test_splitmix64_matches_published_sequence():
    # reference outputs of SplitMix64 seeded with 1234567 (the generator
    # author's test values)
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [int(v) for v in equil.splitmix64_stream(1234567, 5)] == want


def test_signs_are_balanced_and_counter_based():
    s = equil.signs(7, 3, 200000)
    assert set(np.unique(s)) == {-1.0, 1.0}
    assert abs(s.mean()) < 0.01
    # counter-based: a sub-range is the same draw
    np.testing.assert_array_equal(equil.signs(7, 3, 100, offset=50), s[50:150])
    # different blocks differ
    assert (equil.signs(7, 4, 1000) != s[:1000]).mean() > 0.4


def test_probe_estimator_is_unbiased_for_row_and_column_norms():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((40, 25)) * np.exp(rng.uniform(-3, 3, (40, 1)))
    op = scs.Operator(A)
    K = 4000
    r = np.zeros(40)
    c = np.zeros(25)
    for k in range(K):
        r += op.mv(equil.signs(11, k, 25)) ** 2
        c += op.rmv(equil.signs(11, k, 40, 25)) ** 2
    np.testing.assert_allclose(r / K, (A ** 2).sum(1), rtol=0.08)
    np.testing.assert_allclose(c / K, (A ** 2).sum(0), rtol=0.08)


def test_equilibration_balances_rows_and_columns():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((60, 30)) * np.exp(rng.uniform(-4, 4, (60, 1))) * np.exp(rng.uniform(-4, 4, (1, 30)))
    op = scs.Operator(A)
    cone = {"z": 0, "l": 60, "q": []}
    eq = equil.equilibrate(op, cone, np.ones(60), np.ones(30), iters=20, probes=64)
    S = eq["D"][:, None] * A * eq["E"][None, :]
    rn, cn = np.linalg.norm(S, axis=1), np.linalg.norm(S, axis=0)
    before = np.linalg.norm(A, axis=1)
    assert before.max() / before.min() > 1e3
    assert rn.max() / rn.min() < 3.0 and cn.max() / cn.min() < 3.0
    # b^ and c^ are normalised
    assert np.linalg.norm(eq["sigma"] * eq["D"]) == pytest.approx(1.0)
    assert np.linalg.norm(eq["rho"] * eq["E"]) == pytest.approx(1.0)


def test_second_order_cone_rows_share_one_factor():
    rng = np.random.default_rng(2)
    prob = synth.mixed_cone_problem(rng, n=6, soc_sizes=(3, 4), z=1, l=2)
    op = scs.Operator(prob["A"])
    eq = equil.equilibrate(op, prob["cone"], prob["b"], prob["c"], iters=5, probes=4)
    D = eq["D"]
    for lo, hi in equil.soc_blocks(prob["cone"]):
        assert np.all(D[lo:hi] == D[lo])
    assert len(set(np.round(D[:3], 12))) > 1    # the other rows are scaled one by one


def test_equilibrated_lp_solves_the_original_problem():
    rng = np.random.default_rng(3)
    prob = synth.lp(m_d=60, n_x=30, density=0.2, seed=5)
    D = linop.densify(prob["A"]["parts"][0])
    hi = so.linprog(prob["c"], A_ub=D, b_ub=prob["b"][:60], bounds=(0, None), method="highs")
    plain = scs.problem_solve(prob, eps=1e-9, max_iters=200000)
    eqd = scs.problem_solve(prob, eps=1e-9, max_iters=200000, equilibrate=dict(iters=10, probes=8))
    assert eqd["status"] == scs.SOLVED
    assert objective_rel_err(eqd["pobj"], hi.fun) <= 1e-7
    assert objective_rel_err(eqd["pobj"], plain["pobj"]) <= 1e-7
    pri, dual, gap = scs.residuals(scs.Operator(prob["A"]), prob["b"], prob["c"], eqd["x"], eqd["y"], eqd["s"])
    assert max(pri, dual, gap) <= 1e-8
    assert cones.dist_to_dual_cone(eqd["y"], prob["cone"]) <= 1e-9


def test_equilibrated_mixed_cones_and_deconvolution_reach_the_same_optimum():
    rng = np.random.default_rng(4)
    for prob in (synth.mixed_cone_problem(rng, n=8, soc_sizes=(3, 1, 5), z=2, l=4),
                 synth.deconv(n_x=60, L=12, seed=6)):
        plain = scs.problem_solve(prob, eps=1e-10, max_iters=400000)
        eqd = scs.problem_solve(prob, eps=1e-10, max_iters=400000, equilibrate=dict(iters=10, probes=8))
        assert eqd["status"] == scs.SOLVED
        assert objective_rel_err(eqd["pobj"], plain["pobj"]) <= 1e-7
        assert cones.dist_to_cone(eqd["s"], prob["cone"]) <= 1e-8
        assert cones.dist_to_dual_cone(eqd["y"], prob["cone"]) <= 1e-8


@pytest.mark.parametrize("kind", ["infeasible", "unbounded"])
def test_certificates_survive_equilibration(kind):
    rng = np.random.default_rng(300 if kind == "unbounded" else 200)
    D, b_d, c = synth.random_tiny_lp(rng, 3, 3, kind)
    prob = synth.dense_lp(D, b_d, c)
    out = scs.problem_solve(prob, eps=1e-6, eps_infeas=1e-6, max_iters=100000,
                            equilibrate=dict(iters=6, probes=8))
    A = linop.densify(prob["A"])
    if kind == "infeasible":
        assert out["status"] == scs.INFEASIBLE
        assert prob["b"] @ out["y"] == pytest.approx(-1.0)
        assert np.linalg.norm(A.T @ out["y"]) <= 1e-5
        assert cones.dist_to_dual_cone(out["y"], prob["cone"]) <= 1e-9
    else:
        assert out["status"] == scs.UNBOUNDED
        assert prob["c"] @ out["x"] == pytest.approx(-1.0)
        assert np.linalg.norm(A @ out["x"] + out["s"]) <= 1e-5
        assert cones.dist_to_cone(out["s"], prob["cone"]) <= 1e-9


def test_planted_mistake_in_the_scaling_is_caught(monkeypatch):
    """A wrong back-map (dropping sigma from x) makes the equilibrated LP's
    returned point fail the original constraints: the tests above would see it."""
    prob = synth.lp(m_d=40, n_x=20, density=0.3, seed=8)
    eqd = scs.problem_solve(prob, eps=1e-9, max_iters=200000, equilibrate=dict(iters=10, probes=8))
    eq = eqd["equil"]
    tau = eqd["u"][-1]
    n = prob["A"]["n"]
    x_bad = eq["E"] * eqd["u"][:n] / tau          # sigma dropped
    pri_bad = scs.residuals(scs.Operator(prob["A"]), prob["b"], prob["c"], x_bad, eqd["y"], eqd["s"])[0]
    assert abs(eq["sigma"] - 1.0) > 1e-3 and pri_bad > 1e-3


def test_empty_rows_keep_their_scale_and_the_lp_still_solves():
    """A sparse LP with empty rows (120 x 60 at 3% density): the empty rows'
    factor stays 1 (their estimated norm is exactly zero); scaling them up
    instead would shrink sigma by orders of magnitude and stall the solve."""
    prob = synth.lp(m_d=120, n_x=60, density=0.03, seed=170, storage="bf16")
    rp = np.asarray(prob["A"]["parts"][0]["rowptr"])
    empty = np.nonzero(np.diff(rp) == 0)[0]
    assert empty.size > 0
    op = scs.Operator(prob["A"])
    eq = equil.equilibrate(op, prob["cone"], prob["b"], prob["c"], iters=10, probes=8)
    np.testing.assert_array_equal(eq["D"][empty], 1.0)
    out = scs.problem_solve(prob, eps=1e-4, max_iters=40000, linsys="cg", equilibrate=dict(iters=10, probes=8))
    assert out["status"] == scs.SOLVED
