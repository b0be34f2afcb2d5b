"""Pins for the oracle's SCS iteration (Section 5.2 with the published SCS
method it cites).

The optimum is pinned by things that do not depend on the iteration:
brute-force vertex enumeration of tiny LPs, infeasibility/unboundedness
certificates checked against their definitions, scipy's NNLS and HiGHS
solvers, the lasso's subgradient optimality conditions (and the paper's remark
that lam >= ||D^T b||_inf gives x = 0), and the KKT conditions of a mixed-cone
problem.  The subspace step is pinned against a dense solve of the embedding
system (I + Q) u = w."""
import itertools

import numpy as np
import pytest
import scipy.optimize as so

from oracle import cones, linop, scs
from paper_1609_03488_b300 import synth


def _vertex_enum(D, b_d, c):
    """min c^T x s.t. D x <= b_d, x >= 0 by enumerating every vertex."""
    m, n = D.shape
    G = np.vstack([D, -np.eye(n)])
    h = np.concatenate([b_d, np.zeros(n)])
    best = None
    for act in itertools.combinations(range(m + n), n):
        Ga = G[list(act)]
        if abs(np.linalg.det(Ga)) < 1e-12:
            continue
        x = np.linalg.solve(Ga, h[list(act)])
        if np.all(G @ x <= h + 1e-9):
            val = c @ x
            if best is None or val < best[0]:
                best = (val, x)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_tiny_lp_vertex_enumeration(seed):
    rng = np.random.default_rng(100 + seed)
    m, n = int(rng.integers(2, 5)), int(rng.integers(2, 4))
    D, b_d, c = synth.random_tiny_lp(rng, m, n, "feasible")
    best = _vertex_enum(D.astype(np.float32).astype(float), b_d, c)
    assert best is not None
    p = synth.dense_lp(D, b_d, c)
    r = scs.problem_solve(p, eps=1e-9, max_iters=200000)
    assert r["status"] == scs.SOLVED
    assert abs(r["pobj"] - best[0]) <= 1e-6 * (1 + abs(best[0]))


@pytest.mark.parametrize("seed", range(3))
def test_tiny_lp_infeasible_certificate(seed):
    rng = np.random.default_rng(200 + seed)
    D, b_d, c = synth.random_tiny_lp(rng, 3, 3, "infeasible")
    assert _vertex_enum(D.astype(np.float32).astype(float), b_d, c) is None
    p = synth.dense_lp(D, b_d, c)
    r = scs.problem_solve(p, eps=1e-6, max_iters=100000)
    assert r["status"] == scs.INFEASIBLE
    A = linop.densify(p["A"])
    y = r["y"]
    assert abs(p["b"] @ y + 1.0) < 1e-9                      # normalised b^T y = -1
    assert cones.in_dual_cone(y, p["cone"], tol=1e-9)
    assert np.linalg.norm(A.T @ y) <= 1e-6


@pytest.mark.parametrize("seed", range(3))
def test_tiny_lp_unbounded_certificate(seed):
    rng = np.random.default_rng(300 + seed)
    D, b_d, c = synth.random_tiny_lp(rng, 3, 3, "unbounded")
    p = synth.dense_lp(D, b_d, c)
    r = scs.problem_solve(p, eps=1e-6, max_iters=100000)
    assert r["status"] == scs.UNBOUNDED
    A = linop.densify(p["A"])
    x, s = r["x"], r["s"]
    assert abs(p["c"] @ x + 1.0) < 1e-9                      # normalised c^T x = -1
    assert np.linalg.norm(A @ x + s) <= 1e-6
    assert cones.dist_to_cone(s, p["cone"]) <= 1e-6


def test_subspace_step_solves_embedding_system():
    rng = np.random.default_rng(9)
    m, n = 9, 5
    Am = rng.standard_normal((m, n))
    b, c = rng.standard_normal(m), rng.standard_normal(n)
    op = scs.Operator(Am)
    ls = scs._LinSys(op, "direct")
    g_x, g_y, hg = scs.setup(op, b, c, ls)
    Q = np.zeros((n + m + 1, n + m + 1))
    Q[:n, n:n + m] = Am.T
    Q[:n, -1] = c
    Q[n:n + m, :n] = -Am
    Q[n:n + m, -1] = b
    Q[-1, :n] = -c
    Q[-1, n:n + m] = -b
    for _ in range(5):
        w = rng.standard_normal(n + m + 1)
        zx = ls.exact(w[:n] - Am.T @ w[n:n + m])
        ut = scs.subspace_step(op, b, c, g_x, g_y, hg, w, zx)
        np.testing.assert_allclose(ut, np.linalg.solve(np.eye(n + m + 1) + Q, w), rtol=1e-10, atol=1e-12)


def test_cg_mode_with_exact_steps_reproduces_direct_trajectory():
    p = synth.deconv(n_x=30, L=6, seed=4)
    n = p["A"]["n"]
    rd = scs.problem_solve(p, max_iters=15, check_interval=1000, trajectory=15)
    rc = scs.problem_solve(p, max_iters=15, check_interval=1000, trajectory=15,
                           linsys="cg", cg_fixed_steps=n)
    np.testing.assert_allclose(rc["traj_u"], rd["traj_u"], rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(rc["traj_v"], rd["traj_v"], rtol=1e-7, atol=1e-9)


def test_deconv_matches_nnls():
    p = synth.deconv(n_x=120, L=12, seed=2)
    K = linop.densify(p["A"]["parts"][2]["parts"][0]["parts"][0])
    b_obs = p["meta"]["b_obs"]
    x_nn, rnorm = so.nnls(K, b_obs)
    r = scs.problem_solve(p, eps=1e-8, max_iters=100000)
    assert r["status"] == scs.SOLVED
    assert abs(r["pobj"] - rnorm) <= 1e-6 * (1 + rnorm)
    x = np.maximum(r["x"][:-1], 0)
    # NNLS KKT at the returned point: x >= 0, gradient >= 0 off the support
    grad = K.T @ (K @ x - b_obs)
    assert np.all(grad >= -1e-5)
    assert abs(np.linalg.norm(K @ x - b_obs) - rnorm) <= 1e-6


def test_lasso_subgradient_conditions():
    p = synth.lasso(m_d=150, p=60, seed=5)
    D, bo, lam = p["meta"]["D"].astype(float), p["meta"]["b_obs"], p["meta"]["lam"]
    r = scs.problem_solve(p, eps=1e-9, max_iters=100000)
    assert r["status"] == scs.SOLVED
    x = r["x"][:60]
    g = D.T @ (D @ x - bo)
    on = np.abs(x) > 1e-6
    assert np.all(np.abs(g[~on]) <= lam * (1 + 1e-6))
    np.testing.assert_allclose(g[on], -lam * np.sign(x[on]), atol=1e-6 * lam)
    obj = 0.5 * np.sum((D @ x - bo) ** 2) + lam * np.abs(x).sum()
    assert abs(obj - r["pobj"]) <= 1e-6 * (1 + obj)


def test_lasso_zero_solution_above_lambda_max():
    p = synth.lasso(m_d=80, p=30, seed=6, lam_frac=1.05)
    r = scs.problem_solve(p, eps=1e-9, max_iters=100000)
    assert r["status"] == scs.SOLVED
    assert np.abs(r["x"][:30]).max() <= 1e-7


def test_sparse_lp_matches_highs():
    p = synth.lp(m_d=80, n_x=40, density=0.2, seed=12)
    D = linop.densify(p["A"]["parts"][0])
    ref = so.linprog(p["c"], A_ub=D, b_ub=p["b"][:80], bounds=(0, None), method="highs")
    r = scs.problem_solve(p, eps=1e-8, max_iters=400000)
    assert r["status"] == scs.SOLVED
    assert abs(r["pobj"] - ref.fun) <= 1e-6 * (1 + abs(ref.fun))


@pytest.mark.parametrize("seed", range(3))
def test_mixed_cone_kkt(seed):
    rng = np.random.default_rng(400 + seed)
    p = synth.mixed_cone_problem(rng)
    r = scs.problem_solve(p, eps=1e-9, max_iters=200000)
    assert r["status"] == scs.SOLVED
    A = linop.densify(p["A"])
    x, y, s = r["x"], r["y"], r["s"]
    assert np.linalg.norm(A @ x + s - p["b"]) <= 1e-7 * (1 + np.linalg.norm(p["b"]))
    assert np.linalg.norm(A.T @ y + p["c"]) <= 1e-7 * (1 + np.linalg.norm(p["c"]))
    assert cones.dist_to_cone(s, p["cone"]) <= 1e-7
    assert cones.dist_to_dual_cone(y, p["cone"]) <= 1e-7
    assert abs(s @ y) <= 1e-6
    assert abs(p["c"] @ x + p["b"] @ y) <= 1e-6 * (1 + abs(p["c"] @ x))


def test_planted_sign_error_is_caught(monkeypatch):
    """A wrong sign in the SOC projection must break the KKT pin."""
    def bad_soc(v):
        t, z = v[0], v[1:]
        r = np.linalg.norm(z)
        if r <= t:
            return v.copy()
        if r <= -t:
            return np.zeros_like(v)
        a = 0.5 * (t - r)                     # planted: should be t + r
        return np.concatenate([[a], (a / r) * z])

    rng = np.random.default_rng(400)
    p = synth.mixed_cone_problem(rng)
    monkeypatch.setattr(cones, "proj_soc", bad_soc)
    with np.errstate(all="ignore"):
        r = scs.problem_solve(p, eps=1e-9, max_iters=3000)
    A = linop.densify(p["A"])
    with np.errstate(all="ignore"):
        ok = (r["status"] == scs.SOLVED
                  and cones.dist_to_dual_cone(r["y"], p["cone"]) <= 1e-7
              and np.linalg.norm(A.T @ r["y"] + p["c"]) <= 1e-7 * (1 + np.linalg.norm(p["c"])))
    assert not ok
