"""The SCS iteration in FP64 (test infrastructure).

Section 5.2 solves its cone programs with SCS, describing it only as an
iteration that alternates a projection onto a linear subspace (a linear
system solved by the CG method of Section 4.2) and a projection onto a convex
cone; the iteration itself is in the SCS paper the authors cite (O'Donoghue,
Chu, Parikh, Boyd, "Conic optimization via operator splitting and homogeneous
self-dual embedding", 2016).  This module restates that published method in
the order it is defined there.  Readings where the paper is silent are marked
"reading" and listed with the library's design notes.

Problem (Section 2.1, with the sign of the constraint written as the SCS
paper does)::

    minimise c^T x  s.t.  A x + s = b,  s in K          (dual: max -b^T y
                                                        s.t. A^T y + c = 0,
                                                        y in K*)

Homogeneous self-dual embedding: ``u = (x, y, tau)``, ``v = (r, s, kappa)``,
``Q = [[0, A^T, c], [-A, 0, b], [-c^T, -b^T, 0]]``, ``C = R^n x K* x R_+``.
One iteration, with relaxation ``alpha``::

    u~      = (I + Q)^{-1} (u + v)
    u_hat   = alpha u~ + (1 - alpha) u
    u+      = Pi_C(u_hat - v)
    v+      = v - u_hat + u+

``(I + Q)^{-1} w`` is computed through ``M = [[I, A^T], [-A, I]]`` and
``h = (c, b)``: ``z = M^{-1} w_xy`` (``(I + A^T A) z_x = w_x - A^T w_y``,
``z_y = w_y + A z_x``), ``g = M^{-1} h`` once at setup, then
``u~_tau = (w_tau + h^T z) / (1 + h^T g)`` and ``u~_xy = z - u~_tau g``.
"""
from __future__ import annotations

import time

import numpy as np
import scipy.linalg as sla

from . import cg as cg_mod
from . import cones, equil as equil_mod, linop

SOLVED, INFEASIBLE, UNBOUNDED, MAX_ITERS, NUMERICAL = 0, 1, 2, 3, 4
STATUS_NAMES = {SOLVED: "solved", INFEASIBLE: "infeasible", UNBOUNDED: "unbounded",
                MAX_ITERS: "max_iters", NUMERICAL: "numerical"}


class Operator:
    """``A`` either as an explicit float64 matrix or as an operator tree."""

    def __init__(self, A):
        if isinstance(A, dict):
            self.tree = A
            self.m, self.n = A["m"], A["n"]
            self._dense = None
        else:
            self.tree = None
            self._dense = np.asarray(A, dtype=np.float64)
            self.m, self.n = self._dense.shape

    def dense(self):
        if self._dense is None:
            self._dense = linop.densify(self.tree)
        return self._dense

    def mv(self, x):
        if self._dense is not None:
            return self._dense @ x
        return linop.apply(self.tree, x)

    def rmv(self, y):
        if self._dense is not None:
            return self._dense.T @ y
        return linop.apply(self.tree, y, adjoint=True)


def residuals(A, b, c, x, y, s):
    """The termination quantities of the SCS paper at a candidate point
    (reading: l2 norms, relative to ``1 + ||b||`` / ``1 + ||c||``)::

        pri  = ||A x + s - b|| / (1 + ||b||)
        dual = ||A^T y + c||   / (1 + ||c||)
        gap  = |c^T x + b^T y| / (1 + |c^T x| + |b^T y|)
    """
    op = A if isinstance(A, Operator) else Operator(A)
    cx, by = float(c @ x), float(b @ y)
    pri = np.linalg.norm(op.mv(x) + s - b) / (1.0 + np.linalg.norm(b))
    dual = np.linalg.norm(op.rmv(y) + c) / (1.0 + np.linalg.norm(c))
    gap = abs(cx + by) / (1.0 + abs(cx) + abs(by))
    return float(pri), float(dual), float(gap)


class _LinSys:
    """Solver for ``(I + A^T A) z_x = rhs``: dense Cholesky ("direct") or the
    CG recurrence of Section 4.2 warm-started at the previous solution."""

    def __init__(self, op, mode):
        self.op, self.mode = op, mode
        if mode == "direct":
            Ad = op.dense()
            G = np.eye(op.n) + Ad.T @ Ad
            self.chol = sla.cho_factor(G, lower=True)

    def gram(self, p):
        return p + self.op.rmv(self.op.mv(p))

    def exact(self, rhs):
        if self.mode == "direct":
            return sla.cho_solve(self.chol, rhs)
        z, _, _ = cg_mod.cg_recurrence(self.gram, rhs, np.zeros_like(rhs),
                                       stop_abs=1e-13 * float(np.linalg.norm(rhs)),
                                       max_steps=100000)
        return z


def subspace_step(op, b, c, g_x, g_y, hg, w, zx, azx=None):
    """``u~ = (I + Q)^{-1} w`` given ``z_x`` solving
    ``(I + A^T A) z_x = w_x - A^T w_y``::

        z_y    = w_y + A z_x
        u~_tau = (w_tau + c^T z_x + b^T z_y) / (1 + h^T g)
        u~_xy  = z - u~_tau g

    ``azx``: the value to use for ``A z_x`` (the carried one of the
    refinement mode) instead of applying ``A``.
    """
    n, m = op.n, op.m
    w_y, w_tau = w[n:n + m], w[-1]
    zy = w_y + (op.mv(zx) if azx is None else azx)
    ut_tau = (w_tau + c @ zx + b @ zy) / (1.0 + hg)
    return np.concatenate([zx - ut_tau * g_x, zy - ut_tau * g_y, [ut_tau]])


def cg_carried(inner, rhs, zx, az, gz, stop_abs, max_steps, fixed_steps=None):
    """The CG recurrence of Section 4.2 for ``(I + A^T A) z = rhs`` from
    ``z = zx`` in the mixed-precision refinement mode (reading): ``az`` and
    ``gz`` are the values carried for ``A zx`` and ``A^T A zx`` (exact after a
    refresh), the initial residual is ``rhs - zx - gz``, and every step applies
    the inner operand ``A'`` (a lower-precision copy of ``A``)::

        t = A' p;  q = p + A'^T t;  a = r^T r / p^T q
        zx += a p;  r -= a q;  az += a t;  gz += a A'^T t

    Stops as ``cg.cg_recurrence`` does.  Returns ``(zx, az, gz, steps)``
    (new arrays)."""
    zx, az, gz = zx.copy(), az.copy(), gz.copy()
    r = rhs - zx - gz
    p = r.copy()
    rr = float(r @ r)
    k = 0
    while True:
        if fixed_steps is not None:
            if k >= fixed_steps:
                break
        elif not (np.sqrt(rr) > stop_abs and k < max_steps):
            break
        t = inner.mv(p)
        atat = inner.rmv(t)
        q = p + atat
        pq = float(p @ q)
        a = rr / pq if pq > 0 else 0.0
        zx += a * p
        r -= a * q
        az += a * t
        gz += a * atat
        rr_new = float(r @ r)
        beta = rr_new / rr if rr > 0 else 0.0
        p = r + beta * p
        rr = rr_new
        k += 1
    return zx, az, gz, k


REFINE_REFRESH = 50   # iterations between exact A z_x, A^T A z_x in refinement mode (reading)


def setup(op, b, c, ls):
    """``g = M^{-1} h`` with ``h = (c, b)`` and ``h^T g``."""
    g_x = ls.exact(c - op.rmv(b))
    g_y = b + op.mv(g_x)
    return g_x, g_y, float(c @ g_x + b @ g_y)


def solve(A, b, c, cone, *, eps=1e-4, eps_infeas=None, alpha=1.5, max_iters=100000,
          check_interval=10, linsys="direct", cg_fixed_steps=None, cg_max_steps=50,
          cg_tol_rel=1.0, cg_tol_exp=1.5, cg_tol_min=1e-12, trajectory=0, equil=None,
          inner=None, refresh_interval=REFINE_REFRESH):
    """Run SCS on ``min c^T x s.t. A x + s = b, s in K`` in float64.

    ``linsys="direct"`` solves the subspace step exactly (Cholesky of
    ``I + A^T A``); ``linsys="cg"`` uses CG warm-started at the previous
    ``z_x`` with threshold ``max(cg_tol_min, cg_tol_rel ||rhs|| (k+1)^-cg_tol_exp)``
    at iteration k = 0, 1, ... (reading), or exactly ``cg_fixed_steps`` steps.

    Starting point ``u = v = (0, 0, 1)`` (reading).  Every ``check_interval``
    iterations and at the last one, the point ``x = u_x/tau, y = u_y/tau,
    s = v_s/tau`` is tested with ``residuals``; failing that, the
    certificates (reading)::

        infeasible  if -b^T u_y > 0 and ||A^T u_y|| <= eps_infeas (-b^T u_y)
        unbounded   if -c^T u_x > 0 and ||A u_x + v_s|| <= eps_infeas (-c^T u_x)

    ``equil`` (from ``equil.equilibrate``: ``D, E, sigma, rho``) runs the
    iteration on the scaled data ``A^ = D A E``, ``b^ = sigma D b``,
    ``c^ = rho E c``; every test above is then made on the original problem at
    the point mapped back (``x = E x^ / sigma``, ``s = s^ / (sigma D)``,
    ``y = D y^ / rho``; the certificate tests are invariant to the common
    factors), and the point returned is the original one.  ``u``, ``v`` and the
    trajectory stay in the scaled coordinates.

    ``inner`` (an ``Operator`` or operator tree of ``A``'s shape, normally
    ``A`` stored in BF16 or FP8) turns on mixed-precision refinement
    (reading; needs ``linsys="cg"``): the CG steps apply ``inner`` through
    ``cg_carried``, which carries ``A z_x`` and ``A^T A z_x`` along, while the
    right-hand side ``w_x - A^T w_y``, the setup, the termination tests and,
    every ``refresh_interval`` iterations, an exact recomputation of the two
    carried vectors use ``A``.  Both sides of the first CG residual then agree
    with ``A`` up to the drift since the last refresh, so the fixed points are
    those of the problem with ``A``.  (With ``equil``, ``inner`` is scaled by
    the same ``D``, ``E``.)

    Returns a dict with ``x, y, s, status, iters, pobj, dobj, pri, dual, gap,
    u, v, cg_steps``, the wall times ``t_setup`` / ``t_iter`` of the setup and
    of the iterations, and, if ``trajectory`` > 0, the first ``trajectory``
    iterates ``traj_u``/``traj_v``.
    """
    op0 = A if isinstance(A, Operator) else Operator(A)
    m, n = op0.m, op0.n
    b0 = np.asarray(b, dtype=np.float64)
    c0 = np.asarray(c, dtype=np.float64)
    if equil is None:
        Dv, Ev, sigma, rho = np.ones(m), np.ones(n), 1.0, 1.0
        op, b, c = op0, b0, c0
    else:
        Dv, Ev, sigma, rho = equil["D"], equil["E"], float(equil["sigma"]), float(equil["rho"])
        op = equil_mod.ScaledOperator(op0, Dv, Ev)
        b, c = sigma * Dv * b0, rho * Ev * c0
    back = (op0, b0, c0, Dv, Ev, sigma, rho)
    if eps_infeas is None:
        eps_infeas = eps
    opi = None
    if inner is not None:
        if linsys != "cg":
            raise ValueError("refinement (inner) needs linsys='cg'")
        opi = inner if isinstance(inner, Operator) else Operator(inner)
        if (opi.m, opi.n) != (m, n):
            raise ValueError("inner operator shape differs from A's")
        if equil is not None:
            opi = equil_mod.ScaledOperator(opi, Dv, Ev)
    t0 = time.perf_counter()
    ls = _LinSys(op, "direct" if linsys == "direct" else "cg")

    g_x, g_y, hg = setup(op, b, c, ls)
    t1 = time.perf_counter()

    u = np.zeros(n + m + 1)
    v = np.zeros(n + m + 1)
    u[-1] = 1.0
    v[-1] = 1.0
    zx = np.zeros(n)
    az, gz = np.zeros(m), np.zeros(n)     # carried A z_x, A^T A z_x (refinement)
    traj_u, traj_v = [], []
    cg_steps = 0
    status = MAX_ITERS
    res = (np.inf, np.inf, np.inf)
    it = 0
    for k in range(max_iters):
        w = u + v
        w_x, w_y = w[:n], w[n:n + m]
        rhs = w_x - op.rmv(w_y)
        if linsys == "direct":
            zx = ls.exact(rhs)
        else:
            thr = max(cg_tol_min,
                      cg_tol_rel * float(np.linalg.norm(rhs)) * (k + 1.0) ** (-cg_tol_exp))
            if opi is None:
                zx, steps, _ = cg_mod.cg_recurrence(ls.gram, rhs, zx, stop_abs=thr,
                                                    max_steps=cg_max_steps,
                                                    fixed_steps=cg_fixed_steps)
            else:
                zx, az, gz, steps = cg_carried(opi, rhs, zx, az, gz, thr, cg_max_steps,
                                               cg_fixed_steps)
            cg_steps += steps
        ut = subspace_step(op, b, c, g_x, g_y, hg, w, zx, None if opi is None else az)
        u_hat = alpha * ut + (1.0 - alpha) * u
        pre = u_hat - v
        u_new = np.empty_like(u)
        u_new[:n] = pre[:n]
        u_new[n:n + m] = cones.proj_dual_cone(pre[n:n + m], cone)
        u_new[-1] = max(pre[-1], 0.0)
        v = v - u_hat + u_new
        u = u_new
        it = k + 1
        if k < trajectory:
            traj_u.append(u.copy())
            traj_v.append(v.copy())
        if not np.all(np.isfinite(u)) or not np.all(np.isfinite(v)):
            status = NUMERICAL
            break
        if it % check_interval == 0 or it == max_iters:
            st, res = _check(back, u, v, n, m, eps, eps_infeas)
            if st is not None:
                status = st
                break
        if opi is not None and it % refresh_interval == 0:
            az = op.mv(zx)
            gz = op.rmv(az)

    t2 = time.perf_counter()
    tau = u[-1]
    # the point in the original coordinates (identity maps without equil)
    xo, yo, so = Ev * u[:n] / sigma, Dv * u[n:n + m] / rho, v[n:n + m] / (sigma * Dv)
    x = xo / tau if tau > 0 else np.full(n, np.nan)
    y = yo / tau if tau > 0 else np.full(m, np.nan)
    s = so / tau if tau > 0 else np.full(m, np.nan)
    if status == INFEASIBLE:
        d = -float(b0 @ yo)
        x, s, y = np.full(n, np.nan), np.full(m, np.nan), yo / d
    elif status == UNBOUNDED:
        d = -float(c0 @ xo)
        x, s, y = xo / d, so / d, np.full(m, np.nan)
    if status in (SOLVED, MAX_ITERS) and tau > 0:
        res = residuals(op0, b0, c0, x, y, s)
    out = {"x": x, "y": y, "s": s, "status": status, "iters": it,
           "pobj": float(c0 @ x), "dobj": float(-(b0 @ y)),
           "pri": res[0], "dual": res[1], "gap": res[2],
           "u": u, "v": v, "cg_steps": cg_steps, "g_x": g_x, "g_y": g_y, "hg": hg,
           "t_setup": t1 - t0, "t_iter": t2 - t1}
    if trajectory:
        out["traj_u"] = np.array(traj_u)
        out["traj_v"] = np.array(traj_v)
    return out


def _check(back, u, v, n, m, eps, eps_infeas):
    """Termination and certificate tests on the original problem at the
    point the iterate maps back to."""
    op, b, c, Dv, Ev, sigma, rho = back
    tau = u[-1]
    ux = Ev * u[:n] / sigma
    uy = Dv * u[n:n + m] / rho
    vs = v[n:n + m] / (sigma * Dv)
    if tau > 0:
        res = residuals(op, b, c, ux / tau, uy / tau, vs / tau)
        if max(res) <= eps:
            return SOLVED, res
    else:
        res = (np.inf, np.inf, np.inf)
    bty = float(b @ uy)
    if -bty > 0 and np.linalg.norm(op.rmv(uy)) <= eps_infeas * (-bty):
        return INFEASIBLE, res
    ctx = float(c @ ux)
    if -ctx > 0 and np.linalg.norm(op.mv(ux) + vs) <= eps_infeas * (-ctx):
        return UNBOUNDED, res
    return None, res


def problem_solve(prob, equilibrate=None, **kw):
    """``solve`` on a generator problem dict (uses its operator tree).
    ``equilibrate``: None, or a dict of ``equil.equilibrate`` keyword
    arguments (``iters``, ``probes``, ``seed``) to scale the data first; the
    scalings are returned under ``"equil"``.  ``inner`` may be given as an
    operator tree (the refinement mode of ``solve``)."""
    if equilibrate is None:
        return solve(prob["A"], prob["b"], prob["c"], prob["cone"], **kw)
    op = Operator(prob["A"])
    eq = equil_mod.equilibrate(op, prob["cone"], prob["b"], prob["c"], **equilibrate)
    out = solve(op, prob["b"], prob["c"], prob["cone"], equil=eq, **kw)
    out["equil"] = eq
    return out
