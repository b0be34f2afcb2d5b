"""Pins for the oracle's CG (Section 4.2) on the regularized least-squares
problem of Section 5.1, whose solution has the closed form
x* = (lam I + A^T A)^{-1} A^T b; the stop rule is the paper's
||(lam I + A^T A) x - A^T b|| <= 1e-8 ||A^T b||."""
import numpy as np
import pytest

from oracle import cg, linop
from paper_1609_03488_b300 import synth


def _ops(rng, n):
    dense = synth.dense(rng.standard_normal((2 * n, n)).astype(np.float32))
    rp, col, val = synth.random_csr(rng, 2 * n, n, 0.05)
    sparse = synth.csr(2 * n, n, rp, col, val)
    conv = synth.conv1d(synth.gaussian_kernel(n, n / 10.0), n)
    return {"dense": dense, "sparse": sparse, "conv": conv}


@pytest.mark.parametrize("kind", ["dense", "sparse", "conv"])
def test_regularized_ls_closed_form(kind):
    rng = np.random.default_rng(11)
    n, lam = 120, 0.5
    op = _ops(rng, n)[kind]
    A = linop.densify(op)
    xhat = rng.standard_normal(n)
    b = A @ xhat + 0.01 * rng.standard_normal(A.shape[0])
    Atb = A.T @ b
    x_star = np.linalg.solve(lam * np.eye(n) + A.T @ A, Atb)

    def G(p):
        return lam * p + linop.apply(op, linop.apply(op, p), adjoint=True)

    x, k, rr = cg.cg_solve(G, Atb, np.zeros(n), tol=1e-8)
    assert np.linalg.norm(G(x) - Atb) <= 1e-8 * np.linalg.norm(Atb) * 1.0001
    assert np.sqrt(rr) <= 1e-8 * np.linalg.norm(Atb)
    cond = np.linalg.cond(lam * np.eye(n) + A.T @ A)
    assert np.linalg.norm(x - x_star) <= 1e-8 * cond * np.linalg.norm(x_star) * 10
    assert 0 < k <= n


def test_cg_finite_termination():
    rng = np.random.default_rng(5)
    n = 8
    B = rng.standard_normal((n, n))
    S = B @ B.T + n * np.eye(n)
    rhs = rng.standard_normal(n)
    x, k, _ = cg.cg_recurrence(lambda p: S @ p, rhs, np.zeros(n), fixed_steps=n)
    assert k == n
    np.testing.assert_allclose(x, np.linalg.solve(S, rhs), rtol=1e-9)


def test_cg_zero_rhs_and_warm_start_exact():
    S = np.diag([1.0, 2.0, 3.0])
    x, k, rr = cg.cg_recurrence(lambda p: S @ p, np.zeros(3), np.zeros(3), fixed_steps=3)
    assert k == 3 and rr == 0.0 and not x.any()
    xs = np.array([1.0, 1.0, 1.0])
    x, k, rr = cg.cg_recurrence(lambda p: S @ p, S @ xs, xs, stop_abs=1e-12)
    assert k == 0 and np.all(x == xs)
