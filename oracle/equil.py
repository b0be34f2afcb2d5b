"""Matrix-free data equilibration for the SCS iteration, in FP64 (test
infrastructure).

Section 3 of the paper notes that forward and adjoint evaluations of the
operator are all a solver needs, "even" to precondition a problem, citing
stochastic matrix-free equilibration (Diamond and Boyd).  This module is the
reading taken here (see the design notes): diagonal scalings ``D`` (rows)
and ``E`` (columns) found with operator applications only.

* Squared row norms of ``D A E`` are estimated with random sign vectors
  ``s`` (entries +-1): ``E[((D A E) s)_i^2] = sum_j (D A E)_ij^2``; squared
  column norms likewise with ``(D A E)^T w``.  Each iteration averages
  ``probes`` such products.
* Ruiz-style step: ``D_i <- D_i / r_i^(1/4)``, ``E_j <- E_j / c_j^(1/4)`` (each
  row / column divided by the square root of its estimated norm), the
  cumulative factors clipped to [1e-4, 1e4]; a row or column whose
  estimated squared norm is zero (an empty row of a sparse operator) keeps
  its factor, as scaling it would only inflate ``b``.  Rows of one second-order cone
  share one factor (the block's mean squared norm): a positive multiple of
  the cone is the cone, a general diagonal scaling of it is not.
* Then ``b^ = sigma D b`` and ``c^ = rho E c`` with
  ``sigma = 1 / max(||D b||, 1e-3)``, ``rho = 1 / max(||E c||, 1e-3)``.

The scaled problem ``min c^T x^ s.t. A^ x^ + s^ = b^`` with ``A^ = D A E`` has
the solution ``x = E x^ / sigma``, ``s = s^ / (sigma D)``, ``y = D y^ / rho`` of
the original (``scs.solve(..., equil=...)``).

The random signs come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", 2014) used as a counter-based generator:
the value for counter ``k`` is the SplitMix64 output mixing function applied
to ``seed + (k + 1) * 0x9E3779B97F4A7C15 (mod 2^64)``; its top bit set gives -1.
Probe ``k`` of iteration ``t`` uses counters ``(t * probes + k) * 2^32 + j`` for
the column signs (``j < n``) and ``... + n + i`` for the row signs (``i < m``).
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
SCALE_MIN, SCALE_MAX = 1e-4, 1e4
NORM_FLOOR = 1e-3
ZERO_NORM2 = 1e-18


def splitmix64_mix(z):
    """The SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_stream(seed, count):
    """The first ``count`` outputs of SplitMix64 seeded with ``seed`` (state
    advanced by the golden gamma before each output)."""
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = np.uint64(seed) + k * GAMMA
    return splitmix64_mix(x)


def signs(seed, block, length, offset=0):
    """+-1 for counters ``block * 2^32 + offset + j``, j < length."""
    c = (np.uint64(block) << np.uint64(32)) + np.uint64(offset) + np.arange(length, dtype=np.uint64)
    with np.errstate(over="ignore"):
        v = splitmix64_mix(np.uint64(seed) + (c + np.uint64(1)) * GAMMA)
    return np.where((v >> np.uint64(63)) != 0, -1.0, 1.0)


def soc_blocks(cone):
    """(start, stop) of every second-order cone block."""
    off = int(cone.get("z", 0)) + int(cone.get("l", 0))
    out = []
    for q in cone.get("q", []):
        out.append((off, off + int(q)))
        off += int(q)
    return out


def _step(r):
    """Ruiz factor ``r^(-1/4)``; a row / column whose estimated squared norm
    is zero (<= ZERO_NORM2) has nothing to equalise and keeps its scale."""
    return np.where(r > ZERO_NORM2, 1.0 / np.sqrt(np.sqrt(np.maximum(r, ZERO_NORM2))), 1.0)


def equilibrate(op, cone, b, c, iters=10, probes=8, seed=0x5EED):
    """Row / column scalings of the operator ``op`` (``mv``, ``rmv``, ``m``,
    ``n``) and the b / c factors; returns ``dict(D, E, sigma, rho)``."""
    m, n = op.m, op.n
    D = np.ones(m)
    E = np.ones(n)
    blocks = soc_blocks(cone)
    for t in range(iters):
        r = np.zeros(m)
        cc = np.zeros(n)
        for k in range(probes):
            blk = t * probes + k
            s = signs(seed, blk, n, 0)
            w = signs(seed, blk, m, n)
            r += (D * op.mv(E * s)) ** 2
            cc += (E * op.rmv(D * w)) ** 2
        r /= probes
        cc /= probes
        for lo, hi in blocks:
            r[lo:hi] = r[lo:hi].mean()
        D = np.clip(D * _step(r), SCALE_MIN, SCALE_MAX)
        E = np.clip(E * _step(cc), SCALE_MIN, SCALE_MAX)
    b = np.asarray(b, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    sigma = 1.0 / max(float(np.linalg.norm(D * b)), NORM_FLOOR)
    rho = 1.0 / max(float(np.linalg.norm(E * c)), NORM_FLOOR)
    return {"D": D, "E": E, "sigma": sigma, "rho": rho}


class ScaledOperator:
    """``A^ = D A E`` applied matrix-free."""

    def __init__(self, op, D, E):
        self.op, self.D, self.E = op, D, E
        self.m, self.n = op.m, op.n

    def mv(self, x):
        return self.D * self.op.mv(self.E * x)

    def rmv(self, y):
        return self.E * self.op.rmv(self.D * y)

    def dense(self):
        return self.D[:, None] * self.op.dense() * self.E[None, :]
