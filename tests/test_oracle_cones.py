"""Pins for the oracle's cone projections: the defining optimality
conditions of a Euclidean projection onto a closed convex cone (membership,
Moreau decomposition, orthogonality), idempotence, special cases, and a brute
force minimisation over a fine grid of a 3-D second-order cone."""
import numpy as np
import pytest

from oracle import cones


@pytest.mark.parametrize("q", [2, 3, 10, 200])
def test_soc_projection_optimality(q):
    rng = np.random.default_rng(q)
    for _ in range(200):
        v = rng.standard_normal(q) * rng.uniform(0.1, 10)
        p = cones.proj_soc(v)
        # p in K, p - v in K* (= K), and <p, p - v> = 0  (Moreau)
        assert np.linalg.norm(p[1:]) <= p[0] + 1e-12
        d = p - v
        assert np.linalg.norm(d[1:]) <= d[0] + 1e-12
        assert abs(p @ d) <= 1e-10 * (1 + v @ v)
        # v = Pi_K(v) - Pi_K(-v) for a self-dual cone
        np.testing.assert_allclose(v, p - cones.proj_soc(-v), atol=1e-12)
        np.testing.assert_allclose(cones.proj_soc(p), p, atol=1e-12)


def test_soc_special_cases():
    v = np.array([5.0, 3.0, 4.0])
    np.testing.assert_array_equal(cones.proj_soc(v), v)              # on the boundary
    np.testing.assert_array_equal(cones.proj_soc(np.array([-5.0, 3.0, 4.0])), np.zeros(3))
    np.testing.assert_allclose(cones.proj_soc(np.array([0.0, 3.0, 4.0])), [2.5, 1.5, 2.0])


def test_soc_brute_force_grid():
    rng = np.random.default_rng(7)
    # points of Q^3 parametrised by t >= 0, radius rho <= t, angle phi
    t = np.linspace(0, 4, 161)
    frac = np.linspace(0, 1, 81)
    phi = np.linspace(0, 2 * np.pi, 721)
    T, F, P = np.meshgrid(t, frac, phi, indexing="ij")
    pts = np.stack([T, T * F * np.cos(P), T * F * np.sin(P)], -1).reshape(-1, 3)
    for _ in range(10):
        v = rng.uniform(-2, 2, 3)
        best = pts[np.argmin(((pts - v) ** 2).sum(1))]
        p = cones.proj_soc(v)
        assert np.linalg.norm(p - v) <= np.linalg.norm(best - v) + 1e-12
        assert np.linalg.norm(p - best) < 0.06


def test_product_cone_and_dual():
    rng = np.random.default_rng(3)
    cone = {"z": 2, "l": 3, "q": [3, 4]}
    v = rng.standard_normal(12)
    p = cones.proj_cone(v, cone)
    pd = cones.proj_dual_cone(v, cone)
    assert np.all(p[:2] == 0) and np.all(pd[:2] == v[:2])        # {0} and its dual R^z
    np.testing.assert_array_equal(p[2:5], np.maximum(v[2:5], 0))
    assert cones.in_cone(p, cone) and cones.in_dual_cone(pd, cone)
    # Moreau for the product cone: v = Pi_K(v) - Pi_K*(-v)
    np.testing.assert_allclose(v, p - cones.proj_dual_cone(-v, cone), atol=1e-12)
