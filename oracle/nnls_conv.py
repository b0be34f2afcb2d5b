"""Exact nonnegative least squares for a 1-D convolution, in FP64 (test
infrastructure).

Section 5.3 poses nonnegative deconvolution as

    minimise  ||k * x - b||_2   subject to  x >= 0,

with ``k * x`` the full convolution (output length n + L - 1).  The SCS cone
form of that problem has the optimal value ``t* = sqrt(2 f*)`` with

    f* = min_{x >= 0}  f(x),   f(x) = 1/2 ||K x - b||^2,

so an independent solve of this nonnegative least-squares (NNLS) problem pins
the objective of the cone solver at sizes where a dense SCS oracle is out of
reach (n = 1e6: the explicit K would be 2e6 x 1e6).

Method (not the SCS iteration; nothing here is shared with it):

* ``K`` and ``K^T`` are applied by zero-padded real FFTs (Section 2 names the
  FFT as the fast way to evaluate a convolution): ``K x`` is the first
  n + L - 1 entries of ``irfft(rfft(x) rfft(k))``, ``K^T r`` the first n
  entries of ``irfft(rfft(r) conj(rfft(k)))``, both with a transform length
  of at least n + L - 1 so that nothing wraps around.
* The active-set method of Lawson and Hanson (Solving Least Squares Problems,
  1974, ch. 23): a passive set P of variables that are free to be positive;
  the least-squares problem restricted to P is solved exactly; when that
  solution has entries <= 0, the iterate moves towards it until the first
  passive variable reaches zero, which leaves P; when it is positive it
  becomes the iterate, and variables whose gradient entry is negative join P.
  Two departures from the textbook's one-variable-at-a-time loop, both
  harmless to the fixed point: (i) each outer step adds every variable whose
  gradient entry is negative and smallest within a window of +-w samples
  (w = L/20), instead of only the most negative one; (ii) the restricted
  normal equations ``K_P^T K_P z = K_P^T b`` are solved by a banded Cholesky
  factorisation, because ``(K^T K)_{ij}`` is the kernel's autocorrelation at
  lag |i - j| and vanishes for |i - j| >= L, so ``K_P^T K_P`` is banded when P
  is sorted.
* The result is certified by Lagrangian duality (``certificate``): for any
  ``x >= 0`` and any ``y`` with ``K^T y >= 0``,
  ``D(y) = -1/2 ||y||^2 - b^T y <= f* <= f(x)``.  With ``r = K x - b``,
  ``g = K^T r`` and ``h = K^T K 1 > 0`` (the kernel is nonnegative),
  ``y = r + mu K 1`` with ``mu = max(0, max_i -g_i / h_i)`` is dual feasible,
  so ``[sqrt(2 D(y)), sqrt(2 f(x))]`` brackets ``t*``.  At the exact NNLS
  solution (``g_P = 0``, ``g >= 0`` elsewhere) the bracket closes to
  rounding.

Pins (``tests/test_oracle_nnls.py``): the FFT products against
``numpy.convolve`` / ``numpy.correlate`` and the adjoint identity; the
solution against ``scipy.optimize.nnls`` (a dense Lawson-Hanson) and against
brute force over all supports of a tiny instance; weak duality of the bracket
at arbitrary feasible points; and the stored n = 1e6 optimum re-certified
from its stored support.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft
import scipy.linalg as sla
from scipy.ndimage import minimum_filter1d


class ConvOperator:
    """``K``: the full 1-D convolution with ``kernel`` on R^n, applied by
    zero-padded real FFTs (definition: ``(K x)_i = sum_l k_l x_{i-l}``)."""

    def __init__(self, kernel, n, workers=None):
        self.k = np.asarray(kernel, dtype=np.float64)
        self.L = self.k.size
        self.n = int(n)
        self.m = self.n + self.L - 1
        self.nfft = sfft.next_fast_len(self.m, real=True)
        self.kh = sfft.rfft(self.k, self.nfft)
        self.workers = workers

    def mv(self, x):
        X = sfft.rfft(np.asarray(x, dtype=np.float64), self.nfft, workers=self.workers)
        return sfft.irfft(X * self.kh, self.nfft, workers=self.workers)[:self.m]

    def rmv(self, r):
        R = sfft.rfft(np.asarray(r, dtype=np.float64), self.nfft, workers=self.workers)
        return sfft.irfft(R * np.conj(self.kh), self.nfft, workers=self.workers)[:self.n]

    def gram_band(self):
        """``(K^T K)_{i,j} = a_{|i-j|}``: the kernel's autocorrelation,
        ``a_d = sum_l k_l k_{l+d}`` for d = 0 .. L-1 (zero beyond)."""
        full = np.correlate(self.k, self.k, mode="full")
        return full[self.L - 1:]


def restricted_solve(op, P, Ktb, ac):
    """Solve ``K_P^T K_P z = (K^T b)_P`` exactly for the sorted passive index
    set ``P`` (banded Cholesky; bandwidth = the largest number of passive
    indices after any passive index within L - 1 samples)."""
    idx = np.flatnonzero(P)
    s = idx.size
    if s == 0:
        return idx, np.zeros(0)
    L = op.L
    ends = np.searchsorted(idx, idx + L)          # first passive index at lag >= L
    u = int(np.max(ends - np.arange(s))) - 1
    ab = np.zeros((u + 1, s))                     # upper band storage
    for d in range(u + 1):
        lag = idx[d:] - idx[:s - d]
        ab[u - d, d:] = np.where(lag < L, ac[np.minimum(lag, L - 1)], 0.0)
    z = sla.solveh_banded(ab, Ktb[idx], check_finite=False)
    return idx, z


def certificate(op, b, x):
    """Lagrangian-duality bracket of the NNLS optimum at a point ``x >= 0``
    (derivation in the module docstring).  Returns ``f(x)``, the dual value
    ``D(y)`` of the feasible dual point built from ``x``, the bracket of
    ``t* = sqrt(2 f*)``, and the KKT residual ``||x - max(0, x - g)||_inf``."""
    x = np.asarray(x, dtype=np.float64)
    if np.any(x < 0):
        raise ValueError("certificate needs x >= 0")
    r = op.mv(x) - b
    g = op.rmv(r)
    f = 0.5 * float(r @ r)
    ones = np.ones(op.n)
    k1 = op.mv(ones)
    h = op.rmv(k1)
    if np.any(h <= 0):
        raise ValueError("K^T K 1 must be positive (nonnegative kernel)")
    mu = max(0.0, float(np.max(-g / h)))
    y = r + mu * k1
    D = -0.5 * float(y @ y) - float(b @ y)
    kkt = float(np.max(np.abs(x - np.maximum(0.0, x - g)))) if x.size else 0.0
    return {"f": f, "dual": D, "gap": f - D, "mu": mu,
            "t_lo": float(np.sqrt(2.0 * max(D, 0.0))), "t_hi": float(np.sqrt(2.0 * f)),
            "kkt_inf": kkt, "grad_min": float(g.min()) if g.size else 0.0}


def nnls_conv(kernel, b, n, rel_gap=1e-12, max_outer=2000, max_inner=1000, workers=None):
    """Exact ``argmin_{x >= 0} 1/2 ||k * x - b||^2`` by the active-set method
    described in the module docstring.  Stops when the duality bracket's
    relative width ``(f - D)/f`` is at most ``rel_gap`` (or no variable has a
    negative gradient entry).  Returns ``(x, info)`` where ``info`` holds the
    certificate and the step counts."""
    op = ConvOperator(kernel, n, workers=workers)
    b = np.asarray(b, dtype=np.float64)
    if b.size != op.m:
        raise ValueError("b must have n + L - 1 entries")
    if np.any(op.k < 0):
        raise ValueError("the duality certificate assumes a nonnegative kernel")
    ac = op.gram_band()
    Ktb = op.rmv(b)
    gscale = max(float(np.max(np.abs(Ktb))), 1e-300)
    w = max(1, op.L // 20)
    x = np.zeros(op.n)
    P = np.zeros(op.n, dtype=bool)
    g = -Ktb
    outer = inner_total = 0
    cert = None
    for outer in range(1, max_outer + 1):
        # variables leaving the active set: negative gradient entries that are
        # the smallest within +-w samples
        win_min = minimum_filter1d(g, 2 * w + 1, mode="nearest")
        cand = (~P) & (g < -1e-14 * gscale) & (g <= win_min)
        if not cand.any():
            break
        P |= cand
        for _ in range(max_inner):
            inner_total += 1
            idx, z = restricted_solve(op, P, Ktb, ac)
            if np.all(z > 0):
                x = np.zeros(op.n)
                x[idx] = z
                break
            xs = x[idx]
            neg = z <= 0
            alpha = float(np.min(xs[neg] / (xs[neg] - z[neg])))
            xs = xs + alpha * (z - xs)
            drop = neg & (xs <= 1e-14 * max(float(np.max(np.abs(xs))), 1e-300))
            xs[drop] = 0.0
            x = np.zeros(op.n)
            x[idx] = xs
            P[idx[drop]] = False
        g = op.rmv(op.mv(x) - b)
        if outer % 25 == 0:
            cert = certificate(op, b, x)
            if cert["gap"] <= rel_gap * cert["f"]:
                break
    cert = certificate(op, b, x)
    info = dict(cert, outer=outer, inner=inner_total, support=int(np.count_nonzero(x)),
                converged=bool(cert["gap"] <= rel_gap * max(cert["f"], 1e-300)))
    return x, info


def solve_on_support(kernel, b, n, support, workers=None):
    """The least-squares solution restricted to a given support (zero
    elsewhere), and its certificate: re-derives a stored optimum from its
    support alone."""
    op = ConvOperator(kernel, n, workers=workers)
    P = np.zeros(op.n, dtype=bool)
    P[np.asarray(support, dtype=np.int64)] = True
    idx, z = restricted_solve(op, P, op.rmv(np.asarray(b, dtype=np.float64)), op.gram_band())
    x = np.zeros(op.n)
    x[idx] = z
    return x, certificate(op, np.asarray(b, dtype=np.float64), np.maximum(x, 0.0))
