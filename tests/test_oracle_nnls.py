"""Pins of the exact convolution NNLS (oracle/nnls_conv.py), the independent
FP64 optimum of the nonnegative deconvolution of Section 5.3 at full size.

* the FFT products equal numpy's direct convolution / correlation, and are
  adjoint to each other (asymmetric kernels, so a flipped kernel fails);
* the solution equals scipy.optimize.nnls (a dense Lawson-Hanson) and brute
  force over every support of a tiny instance;
* the duality bracket contains the optimum at arbitrary feasible points
  (weak duality) and closes at the solution;
* planted mistakes in the oracle (a truncated Gram band, a flipped kernel)
  are caught by the scipy comparison;
* the stored n = 1e6 optimum: its instance fingerprint matches the generator,
  and the optimum re-derived from the stored support alone is certified
  within its stored bracket.
"""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.optimize as so

from oracle import linop, nnls_conv
from paper_1609_03488_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "deconv_large_optimum.json")


def _asym_kernel(rng, L):
    k = rng.random(L) ** 2
    k[0] += 0.5                       # clearly asymmetric
    return k / k.sum()


def _dense(kernel, n):
    return linop._dense_conv1d(np.asarray(kernel, dtype=np.float64), n)


def test_fft_products_match_direct_sums_and_are_adjoint():
    rng = np.random.default_rng(11)
    for n, L in ((1, 1), (7, 3), (100, 17), (1000, 1000), (4097, 255)):
        k = _asym_kernel(rng, L)
        op = nnls_conv.ConvOperator(k, n)
        x, r = rng.standard_normal(n), rng.standard_normal(n + L - 1)
        np.testing.assert_allclose(op.mv(x), np.convolve(k, x), rtol=0, atol=1e-12 * np.abs(x).sum())
        np.testing.assert_allclose(op.rmv(r), np.correlate(r, k, mode="valid"), rtol=0,
                                   atol=1e-12 * np.abs(r).sum())
        assert abs(op.mv(x) @ r - x @ op.rmv(r)) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(r) * L


def test_gram_band_is_the_explicit_gram():
    rng = np.random.default_rng(12)
    k = _asym_kernel(rng, 9)
    op = nnls_conv.ConvOperator(k, 30)
    G = _dense(k, 30).T @ _dense(k, 30)
    a = op.gram_band()
    for i in range(30):
        for j in range(30):
            d = abs(i - j)
            np.testing.assert_allclose(G[i, j], a[d] if d < 9 else 0.0, atol=1e-15)


@pytest.mark.parametrize("n,L,seed", [(300, 30, 1), (2000, 100, 1), (500, 120, 7)])
def test_matches_scipy_nnls_on_the_deconvolution_generator(n, L, seed):
    p = synth.deconv(n_x=n, L=L, seed=synth.BASE_SEED + seed)
    k, b = p["meta"]["kernel"], p["meta"]["b_obs"]
    x, info = nnls_conv.nnls_conv(k, b, n)
    xs, rn = so.nnls(_dense(k, n), b, maxiter=100 * n)
    f_star = 0.5 * rn * rn
    assert info["converged"]
    assert abs(info["f"] - f_star) <= 1e-12 * f_star
    assert np.all(x >= 0)
    np.testing.assert_allclose(x, xs, rtol=0, atol=1e-7 * max(1.0, np.abs(xs).max()))
    assert info["t_lo"] <= np.sqrt(2 * f_star) * (1 + 1e-14) and np.sqrt(2 * f_star) <= info["t_hi"] * (1 + 1e-14)


def test_matches_scipy_nnls_with_an_asymmetric_kernel():
    rng = np.random.default_rng(5)
    n, L = 400, 40
    k = _asym_kernel(rng, L)
    b = np.convolve(k, np.maximum(rng.standard_normal(n), 0) * (rng.random(n) < 0.1)) \
        + 0.01 * rng.standard_normal(n + L - 1)
    x, info = nnls_conv.nnls_conv(k, b, n)
    xs, rn = so.nnls(_dense(k, n), b, maxiter=100 * n)
    assert abs(info["f"] - 0.5 * rn * rn) <= 1e-12 * (0.5 * rn * rn)
    np.testing.assert_allclose(x, xs, atol=1e-8)


def test_brute_force_over_all_supports():
    rng = np.random.default_rng(3)
    n, L = 8, 4
    k = _asym_kernel(rng, L)
    K = _dense(k, n)
    for trial in range(4):
        b = rng.standard_normal(n + L - 1)
        best = 0.5 * b @ b                       # x = 0
        for r_ in range(1, n + 1):
            for S in itertools.combinations(range(n), r_):
                z, *_ = np.linalg.lstsq(K[:, S], b, rcond=None)
                if np.all(z >= 0):
                    best = min(best, 0.5 * np.sum((K[:, S] @ z - b) ** 2))
        _, info = nnls_conv.nnls_conv(k, b, n)
        assert abs(info["f"] - best) <= 1e-12 * max(best, 1e-12)


def test_bracket_is_valid_at_any_feasible_point_and_closes_at_the_solution():
    p = synth.deconv(n_x=500, L=50, seed=synth.BASE_SEED + 9)
    k, b = p["meta"]["kernel"], p["meta"]["b_obs"]
    xs, rn = so.nnls(_dense(k, 500), b, maxiter=50000)
    t_star = rn
    op = nnls_conv.ConvOperator(k, 500)
    rng = np.random.default_rng(0)
    for scale in (0.0, 0.1, 1.0, 10.0):
        x = np.maximum(xs + scale * rng.standard_normal(500), 0.0)
        c = nnls_conv.certificate(op, b, x)
        assert c["t_lo"] <= t_star * (1 + 1e-14) and t_star <= c["t_hi"] * (1 + 1e-14), (scale, c)
    c = nnls_conv.certificate(op, b, np.maximum(xs, 0))
    assert c["gap"] <= 1e-9 * c["f"]
    with pytest.raises(ValueError):
        nnls_conv.certificate(op, b, -np.ones(500))


def test_planted_mistakes_are_caught(monkeypatch):
    p = synth.deconv(n_x=600, L=60, seed=synth.BASE_SEED + 1)
    k, b = p["meta"]["kernel"], p["meta"]["b_obs"]
    _, rn = so.nnls(_dense(k, 600), b, maxiter=60000)
    f_star = 0.5 * rn * rn
    # a Gram band missing its last lags: the restricted solves are wrong
    good = nnls_conv.ConvOperator.gram_band
    monkeypatch.setattr(nnls_conv.ConvOperator, "gram_band", lambda self: np.concatenate(
        [good(self)[:self.L // 2], np.zeros(self.L - self.L // 2)]))
    try:
        _, info = nnls_conv.nnls_conv(k, b, 600, max_outer=200)
        assert abs(info["f"] - f_star) > 1e-6 * f_star
    except np.linalg.LinAlgError:
        pass                            # the wrong Gram is not even positive definite
    monkeypatch.setattr(nnls_conv.ConvOperator, "gram_band", good)
    # a flipped kernel (correlation for convolution) on an asymmetric kernel
    rng = np.random.default_rng(8)
    ka = _asym_kernel(rng, 60)
    ba = np.convolve(ka, np.maximum(rng.standard_normal(600), 0)) + 0.01 * rng.standard_normal(659)
    _, rna = so.nnls(_dense(ka, 600), ba, maxiter=60000)
    _, info = nnls_conv.nnls_conv(ka[::-1].copy(), ba, 600)
    assert abs(info["f"] - 0.5 * rna * rna) > 1e-6 * (0.5 * rna * rna)


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="stored optimum not written")
def test_stored_large_optimum_is_certified_from_its_support():
    g = json.load(open(GOLDEN))
    inst = g["instance"]
    p = synth.deconv(**inst)
    k = np.asarray(p["meta"]["kernel"], dtype=np.float64)
    b = np.asarray(p["meta"]["b_obs"], dtype=np.float64)
    fp = g["fingerprint"]
    assert k.sum() == pytest.approx(fp["kernel_sum"], rel=1e-15) and b @ b == pytest.approx(fp["b_obs_sq"], rel=1e-13)
    assert b[0] == fp["b_obs_first"] and b[-1] == fp["b_obs_last"]
    x, c = nnls_conv.solve_on_support(k, b, inst["n_x"], g["support"], workers=os.cpu_count())
    assert np.all(x[g["support"]] > 0)
    # the bracket re-derived here is tight and agrees with the stored one
    assert c["t_hi"] - c["t_lo"] <= 1e-9 * c["t_hi"]
    assert c["t_lo"] <= g["t_hi"] * (1 + 1e-12) and g["t_lo"] <= c["t_hi"] * (1 + 1e-12)
    assert c["kkt_inf"] <= 1e-12
