"""Conjugate gradient, as described in Section 4.2 (test infrastructure).

The paper's ``cg_solve(A, b, x_init, tol)`` runs the classical CG recurrence
(Hestenes-Stiefel) from ``x_init`` and keeps iterating while
``||r||_2 > tol * ||b||_2``; it returns the iterate, the step count and
``||r||^2``.  The same recurrence, with an absolute threshold and a step cap,
is the inner linear-system solver of the SCS iteration (Section 5.2).
"""
from __future__ import annotations

import numpy as np


def cg_recurrence(apply, rhs, x0, stop_abs=0.0, max_steps=10 ** 9, fixed_steps=None):
    """CG on an SPD operator ``apply`` from ``x0``.

    Continues while ``||r|| > stop_abs`` and fewer than ``max_steps`` steps
    were taken; with ``fixed_steps`` it takes exactly that many steps and
    ignores the threshold.  A zero curvature ``p^T A p`` (which only occurs
    when ``r = 0``) takes a zero step.  Returns ``(x, steps, ||r||^2)``.
    """
    x = np.array(x0, dtype=np.float64, copy=True)
    r = np.asarray(rhs, dtype=np.float64) - apply(x)
    p = r.copy()
    rr = float(r @ r)
    k = 0
    while True:
        if fixed_steps is not None:
            if k >= fixed_steps:
                break
        elif not (np.sqrt(rr) > stop_abs and k < max_steps):
            break
        Ap = apply(p)
        pAp = float(p @ Ap)
        a = rr / pAp if pAp > 0 else 0.0
        x += a * p
        r -= a * Ap
        rr_new = float(r @ r)
        beta = rr_new / rr if rr > 0 else 0.0
        p = r + beta * p
        rr = rr_new
        k += 1
    return x, k, rr


def cg_solve(apply, b, x_init, tol=1e-8, max_steps=10 ** 6):
    """Section 4.2's ``cg_solve``: relative stop ``||r|| <= tol ||b||``."""
    b = np.asarray(b, dtype=np.float64)
    return cg_recurrence(apply, b, x_init, stop_abs=tol * float(np.linalg.norm(b)),
                         max_steps=max_steps)
