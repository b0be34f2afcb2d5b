"""Pins for the oracle's structured operators (Section 3.1).

Dense materialisation is checked against independent library routines
(scipy's direct convolutions), against explicit index formulas, and the
matrix-free apply is checked against the materialised matrix and against the
adjoint identity <A x, y> = <x, A^T y>."""
import json
import os

import numpy as np
import pytest
import scipy.signal

from oracle import linop
from paper_1609_03488_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table_sizes.json")


def _rand_tree(rng):
    D = rng.standard_normal((7, 5)).astype(np.float32)
    rp, col, val = synth.random_csr(rng, 6, 5, 0.5)
    k = rng.standard_normal(3).astype(np.float32)
    K2 = rng.standard_normal((2, 3)).astype(np.float32)
    B = rng.standard_normal((2, 3)).astype(np.float32)
    C = rng.standard_normal((3, 2)).astype(np.float32)
    d = rng.standard_normal(5).astype(np.float32)
    return synth.vstack([
        synth.dense(D),
        synth.csr(6, 5, rp, col, val),
        synth.conv1d(k, 5),
        synth.scale(-2.0, synth.diag(5, d)),
        synth.product([synth.dense(rng.standard_normal((4, 7)).astype(np.float32)), synth.dense(D)]),
        synth.opsum([synth.eye(5), synth.adjoint(synth.dense(rng.standard_normal((5, 5)).astype(np.float32)))]),
        synth.hstack([synth.zero(3, 2), synth.dense(rng.standard_normal((3, 3)).astype(np.float32))]),
        synth.blockdiag([synth.dense(B), synth.dense(rng.standard_normal((1, 2)).astype(np.float32))]),
        synth.product([synth.kron(synth.dense(C), synth.dense(B)), synth.dense(rng.standard_normal((6, 5)).astype(np.float32))]),
        synth.conv2d(K2, 1, 5),
    ])


def test_conv1d_dense_matches_scipy():
    rng = np.random.default_rng(0)
    for n, L in [(10, 1), (10, 4), (3, 7), (50, 13)]:
        k = rng.standard_normal(L)
        x = rng.standard_normal(n)
        T = linop.densify(synth.conv1d(k, n))
        np.testing.assert_allclose(T @ x, scipy.signal.convolve(x, k, method="direct"), rtol=1e-6, atol=1e-6)
        # matrix-free
        np.testing.assert_allclose(linop.apply(synth.conv1d(k, n), x), T @ x.astype(np.float64), rtol=1e-6, atol=1e-6)


def test_conv1d_toeplitz_entries():
    k = np.array([1.0, 2.0, 3.0], dtype=np.float32)
    T = linop.densify(synth.conv1d(k, 2))
    np.testing.assert_array_equal(T, np.array([[1, 0], [2, 1], [3, 2], [0, 3]], dtype=float))


def test_conv2d_dense_matches_scipy():
    rng = np.random.default_rng(1)
    K = rng.standard_normal((3, 4)).astype(np.float32)
    X = rng.standard_normal((5, 6))
    T = linop.densify(synth.conv2d(K, 5, 6))
    ref = scipy.signal.convolve2d(X, K.astype(np.float64), mode="full").ravel()
    np.testing.assert_allclose(T @ X.ravel(), ref, rtol=1e-10, atol=1e-10)


def test_kron_vec_identity():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((3, 4)).astype(np.float32)
    B = rng.standard_normal((2, 5)).astype(np.float32)
    X = rng.standard_normal((4, 5))
    op = synth.kron(synth.dense(A), synth.dense(B))
    want = np.einsum("ij,jl,kl->ik", A.astype(float), X, B.astype(float)).ravel()  # A X B^T
    np.testing.assert_allclose(linop.densify(op) @ X.ravel(), want, rtol=1e-10)
    np.testing.assert_allclose(linop.apply(op, X.ravel()), want, rtol=1e-10)


def test_compositions_match_blocks():
    rng = np.random.default_rng(3)
    P = rng.standard_normal((3, 4)).astype(np.float32)
    R = rng.standard_normal((4, 2)).astype(np.float32)
    Pd, Rd = P.astype(float), R.astype(float)
    assert np.allclose(linop.densify(synth.product([synth.dense(P), synth.dense(R)])), Pd @ Rd)
    assert np.allclose(linop.densify(synth.adjoint(synth.dense(P))), Pd.T)
    assert np.allclose(linop.densify(synth.scale(3.0, synth.dense(P))), 3 * Pd)
    V = linop.densify(synth.vstack([synth.dense(P), synth.zero(2, 4)]))
    assert V.shape == (5, 4) and np.allclose(V[:3], Pd) and not V[3:].any()
    H = linop.densify(synth.hstack([synth.dense(P), synth.eye(3)]))
    assert np.allclose(H[:, :4], Pd) and np.allclose(H[:, 4:], np.eye(3))


def test_matrix_free_equals_dense_and_adjoint_identity():
    rng = np.random.default_rng(4)
    op = _rand_tree(rng)
    T = linop.densify(op)
    assert T.shape == (op["m"], op["n"])
    for _ in range(3):
        x = rng.standard_normal(op["n"])
        y = rng.standard_normal(op["m"])
        Ax = linop.apply(op, x)
        ATy = linop.apply(op, y, adjoint=True)
        np.testing.assert_allclose(Ax, T @ x, rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(ATy, T.T @ y, rtol=1e-9, atol=1e-9)
        assert abs(Ax @ y - x @ ATy) <= 1e-9 * (1 + abs(Ax @ y))


def test_paper_problem_sizes():
    g = json.load(open(GOLDEN))
    for case in g["deconv"]["cases"]:
        if case["n_x"] > 1000:
            continue   # densify-free size check below
        p = synth.deconv(n_x=case["n_x"], L=case["n_x"], seed=1)
        assert p["A"]["n"] == case["variables"]
        assert p["A"]["m"] == case["constraints"]
        assert synth.cone_dims(p["cone"]) == case["constraints"]
    big = g["deconv"]["cases"][-1]
    p = synth.deconv(n_x=big["n_x"], L=big["n_x"], seed=1)
    assert (p["A"]["n"], p["A"]["m"]) == (big["variables"], big["constraints"])


@pytest.mark.slow
def test_paper_lasso_size_and_nnz():
    g = json.load(open(GOLDEN))["lasso_dense"]
    p = synth.lasso(m_d=g["m_d"], p=g["p"], seed=1)
    assert p["A"]["n"] == g["variables"]
    assert p["A"]["m"] == g["constraints"]
    assert linop.nnz(p["A"]) == g["nnz"]


def test_paper_convolution_lasso_size():
    g = json.load(open(GOLDEN))["lasso_conv"]
    p = synth.lasso_conv(p=g["p"], L=g["L"], seed=1)
    assert (p["A"]["n"], p["A"]["m"]) == (g["variables"], g["constraints"])
    assert synth.cone_dims(p["cone"]) == g["constraints"]


def test_storage_variants_of_one_tree_keep_their_own_values():
    """Trees that share a leaf's data but store it differently (the float32
    instance and its BF16 / FP8 inner copies) are applied with their own
    dequantised values, whichever was applied first: the oracle's per-leaf
    cache is keyed by the storage."""
    from oracle import quant
    rng = np.random.default_rng(9)
    prob = synth.lasso(m_d=50, p=20, seed=9)
    x = rng.standard_normal(prob["A"]["n"])
    y32 = linop.apply(prob["A"], x)                      # fills the float32 cache first
    for storage in ("bf16", "fp8"):
        t = synth.with_storage(prob["A"], storage)
        D = quant.dense_values(prob["meta"]["D"], storage)
        yq = linop.apply(t, x)
        p = prob["meta"]["p"]
        np.testing.assert_allclose(yq[-50:], -np.sqrt(2.0) * (D @ x[:p]), rtol=1e-12, atol=1e-12)
        assert np.abs(yq - y32).max() > 1e-6
    np.testing.assert_array_equal(linop.apply(prob["A"], x), y32)
    # the convolution method switch changes nothing in the operator
    dec = synth.deconv(n_x=40, L=9, seed=3)
    z = rng.standard_normal(dec["A"]["n"])
    for method in ("direct", "fft"):
        np.testing.assert_array_equal(linop.apply(synth.with_conv_method(dec["A"], method), z),
                                      linop.apply(dec["A"], z))
