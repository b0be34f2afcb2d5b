"""Oracle pins of the lasso variants and the 2-D deconvolution of Sections
5.2 / 2: the oracle's solutions satisfy the problems' own optimality
conditions (lasso: subgradient KKT; nonnegative least squares: agreement
with scipy's NNLS on the explicit operator)."""
import numpy as np
import scipy.optimize as so

from oracle import linop, scs
from paper_1609_03488_b300 import synth


def _lasso_kkt(prob, x, tol):
    D = linop.densify(prob["A"]["parts"][4]["parts"][0]["parts"][0])
    p = prob["meta"]["p"]
    xx = x[:p]
    g = D.T @ (D @ xx - prob["meta"]["b_obs"])
    lam = prob["meta"]["lam"]
    assert np.all(np.abs(g) <= lam * (1 + tol))
    nz = np.abs(xx) > 1e-6
    np.testing.assert_allclose(g[nz], -lam * np.sign(xx[nz]), rtol=tol, atol=tol * lam)


def test_sparse_and_convolution_lasso_kkt():
    # the Gaussian-blur convolution is badly conditioned: plain SCS crawls
    # there, the equilibrated iteration (pinned in test_oracle_equil.py)
    # reaches 1e-8 in ~2e3 iterations
    for prob, eq in ((synth.lasso_sparse(m_d=300, p=150, density=0.05, seed=21), None),
                     (synth.lasso_conv(p=120, L=40, seed=22), dict(iters=10, probes=8))):
        r = scs.problem_solve(prob, eps=1e-8, max_iters=200000, equilibrate=eq)
        assert r["status"] == scs.SOLVED
        _lasso_kkt(prob, r["x"], 1e-3)


def test_deconv2d_matches_nnls():
    prob = synth.deconv2d(h=10, w=9, kh=5, kw=4, seed=23)
    K = linop.densify(prob["A"]["parts"][2]["parts"][0]["parts"][0])
    assert K.shape == ((10 + 5 - 1) * (9 + 4 - 1), 90)
    _, rnorm = so.nnls(K, prob["meta"]["b_obs"], maxiter=20000)
    r = scs.problem_solve(prob, eps=1e-10, max_iters=400000)
    assert r["status"] == scs.SOLVED
    assert abs(r["pobj"] - rnorm) <= 1e-6 * (1 + rnorm)
