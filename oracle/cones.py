"""Euclidean projections onto the cones of the standard form (test
infrastructure).

The paper's experiments canonicalise to the zero, nonnegative and
second-order cones (lasso, Section 5.2; nonnegative deconvolution,
Section 5.3); it gives no projection formulas.  These are the textbook closed
forms:

* zero cone {0}: projection is 0; its dual cone is the whole space, whose
  projection is the identity.
* nonnegative orthant: ``max(v, 0)`` elementwise (self-dual).
* second-order cone Q = {(t, z): ||z||_2 <= t} (self-dual): with ``r = ||z||``,
  ``(t, z)`` if ``r <= t``; ``0`` if ``r <= -t``; otherwise
  ``((t + r)/2) * (1, z / r)``.

Rows are ordered zero, nonnegative, then each SOC block.
"""
from __future__ import annotations

import numpy as np


def proj_nonneg(v):
    return np.maximum(v, 0.0)


def proj_soc(v):
    v = np.asarray(v, dtype=np.float64)
    t, z = v[0], v[1:]
    r = np.linalg.norm(z)
    if r <= t:
        return v.copy()
    if r <= -t:
        return np.zeros_like(v)
    a = 0.5 * (t + r)
    out = np.empty_like(v)
    out[0] = a
    out[1:] = (a / r) * z
    return out


def _segments(cone):
    z = int(cone.get("z", 0))
    l = int(cone.get("l", 0))
    q = [int(s) for s in cone.get("q", [])]
    return z, l, q


def proj_cone(v, cone):
    """Projection onto K = {0}^z x R_+^l x Q^{q_1} x ... ."""
    z, l, q = _segments(cone)
    out = np.empty_like(np.asarray(v, dtype=np.float64))
    out[:z] = 0.0
    out[z:z + l] = proj_nonneg(v[z:z + l])
    off = z + l
    for s in q:
        out[off:off + s] = proj_soc(v[off:off + s])
        off += s
    return out


def proj_dual_cone(v, cone):
    """Projection onto K* = R^z x R_+^l x Q^{q_1} x ... (zero cone's dual is
    the free space; the other cones are self-dual)."""
    z, l, q = _segments(cone)
    out = np.empty_like(np.asarray(v, dtype=np.float64))
    out[:z] = v[:z]
    out[z:z + l] = proj_nonneg(v[z:z + l])
    off = z + l
    for s in q:
        out[off:off + s] = proj_soc(v[off:off + s])
        off += s
    return out


def in_cone(v, cone, tol=1e-9):
    z, l, q = _segments(cone)
    if z and np.max(np.abs(v[:z])) > tol:
        return False
    if l and np.min(v[z:z + l]) < -tol:
        return False
    off = z + l
    for s in q:
        if np.linalg.norm(v[off + 1:off + s]) > v[off] + tol:
            return False
        off += s
    return True


def in_dual_cone(v, cone, tol=1e-9):
    z, l, q = _segments(cone)
    if l and np.min(v[z:z + l]) < -tol:
        return False
    off = z + l
    for s in q:
        if np.linalg.norm(v[off + 1:off + s]) > v[off] + tol:
            return False
        off += s
    return True


def dist_to_cone(v, cone):
    return float(np.linalg.norm(v - proj_cone(v, cone)))


def dist_to_dual_cone(v, cone):
    return float(np.linalg.norm(v - proj_dual_cone(v, cone)))
