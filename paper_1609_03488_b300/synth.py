"""Seeded synthetic cone programs shaped like the paper's workloads.

This module only *describes* inputs: it draws random data and writes each
problem down in the cone standard form (Section 2.1, problem (1), written here
with the sign convention ``A x + s = b, s in K``).  It holds none of the
solver's arithmetic and imports nothing else from this package, so both the
CUDA path and the FP64 oracle can consume the same description.

A problem is a dict::

    {"A": <operator tree>, "b": float64[m], "c": float64[n],
     "cone": {"z": zero rows, "l": nonneg rows, "q": [SOC sizes]},
     "family": ..., "meta": {...}}

An operator tree node is a dict with a ``"kind"`` key:

* leaves: ``dense`` (``data`` float32 m x n row-major, ``storage`` one of
  ``fp32``/``bf16``/``fp8``), ``csr`` (``rowptr``/``col`` int32, ``val``
  float32, ``storage`` ``fp32``/``bf16``), ``conv1d`` (full convolution with
  ``kernel``, input length ``n``), ``conv2d`` (full 2-D convolution of an
  ``h x w`` image with a 2-D ``kernel``), ``diag`` (``d`` or ``None`` for the
  identity), ``zero`` (``m x n``);
* compositions (Section 3.1, structured linear operators): ``vstack``,
  ``hstack``, ``blockdiag``, ``sum``, ``product`` (``parts[0] @ parts[1] @
  ...``), ``scale`` (``alpha * parts[0]``), ``adjoint``, ``kron``
  (``parts[0] (x) parts[1]``, row-major vec).

Rows of ``A`` are ordered zero cone, nonnegative cone, then each second-order
cone; a second-order cone row block ``(t, z)`` means ``||z||_2 <= t``.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20161116


# ---------------------------------------------------------------- tree nodes
def dense(data, storage="fp32"):
    data = np.ascontiguousarray(data, dtype=np.float32)
    return {"kind": "dense", "m": data.shape[0], "n": data.shape[1],
            "data": data, "storage": storage}


def csr(m, n, rowptr, col, val, storage="fp32"):
    return {"kind": "csr", "m": int(m), "n": int(n),
            "rowptr": np.ascontiguousarray(rowptr, dtype=np.int32),
            "col": np.ascontiguousarray(col, dtype=np.int32),
            "val": np.ascontiguousarray(val, dtype=np.float32),
            "storage": storage}


def conv1d(kernel, n, method="auto"):
    """Full 1-D convolution leaf; ``method`` ("auto", "direct", "fft") only
    selects how the library evaluates it."""
    kernel = np.ascontiguousarray(kernel, dtype=np.float32)
    return {"kind": "conv1d", "m": int(n) + kernel.size - 1, "n": int(n),
            "kernel": kernel, "method": method}


def conv2d(kernel, h, w):
    kernel = np.ascontiguousarray(kernel, dtype=np.float32)
    kh, kw = kernel.shape
    return {"kind": "conv2d", "m": (h + kh - 1) * (w + kw - 1), "n": h * w,
            "h": int(h), "w": int(w), "kernel": kernel}


def diag(n, d=None):
    if d is not None:
        d = np.ascontiguousarray(d, dtype=np.float32)
        assert d.size == n
    return {"kind": "diag", "m": int(n), "n": int(n), "d": d}


def eye(n):
    return diag(n, None)


def zero(m, n):
    return {"kind": "zero", "m": int(m), "n": int(n)}


def with_conv_method(tree, method):
    """A copy of an operator tree whose 1-D convolution leaves are evaluated
    by ``method`` ("auto", "direct" or "fft"); same operator."""
    if tree["kind"] == "conv1d":
        return {k: v for k, v in tree.items() if not k.startswith("_")} | {"method": method}
    if "parts" in tree:
        return {**tree, "parts": [with_conv_method(p, method) for p in tree["parts"]]}
    return tree


def with_storage(tree, storage):
    """A copy of an operator tree whose dense and CSR leaves are stored in
    ``storage`` (the data arrays are shared, not copied): the lower-precision
    inner operand of the refinement mode, built from the float32 instance."""
    if tree["kind"] in ("dense", "csr"):
        return {k: v for k, v in tree.items() if not k.startswith("_")} | {"storage": storage}
    if "parts" in tree:
        return {**tree, "parts": [with_storage(p, storage) for p in tree["parts"]]}
    return tree


def scale(alpha, part):
    return {"kind": "scale", "alpha": float(alpha), "parts": [part],
            "m": part["m"], "n": part["n"]}


def adjoint(part):
    return {"kind": "adjoint", "parts": [part], "m": part["n"], "n": part["m"]}


def vstack(parts):
    n = parts[0]["n"]
    assert all(p["n"] == n for p in parts)
    return {"kind": "vstack", "parts": list(parts),
            "m": sum(p["m"] for p in parts), "n": n}


def hstack(parts):
    m = parts[0]["m"]
    assert all(p["m"] == m for p in parts)
    return {"kind": "hstack", "parts": list(parts), "m": m,
            "n": sum(p["n"] for p in parts)}


def blockdiag(parts):
    return {"kind": "blockdiag", "parts": list(parts),
            "m": sum(p["m"] for p in parts), "n": sum(p["n"] for p in parts)}


def opsum(parts):
    m, n = parts[0]["m"], parts[0]["n"]
    assert all(p["m"] == m and p["n"] == n for p in parts)
    return {"kind": "sum", "parts": list(parts), "m": m, "n": n}


def product(parts):
    for a, b in zip(parts[:-1], parts[1:]):
        assert a["n"] == b["m"]
    return {"kind": "product", "parts": list(parts), "m": parts[0]["m"],
            "n": parts[-1]["n"]}


def kron(a, b):
    return {"kind": "kron", "parts": [a, b], "m": a["m"] * b["m"],
            "n": a["n"] * b["n"]}


def cone_dims(cone):
    return int(cone.get("z", 0)) + int(cone.get("l", 0)) + int(sum(cone.get("q", [])))


# ------------------------------------------------------------- random pieces
def rng_for(seed):
    return np.random.default_rng(int(seed))


def gaussian_kernel(L, sigma):
    """Sampled Gaussian of length L centred at (L-1)/2, normalised to sum 1."""
    i = np.arange(L, dtype=np.float64)
    k = np.exp(-((i - (L - 1) / 2.0) ** 2) / (2.0 * sigma * sigma))
    return k / k.sum()


def sparse_nonneg_signal(rng, n, frac):
    """Support drawn uniformly without replacement, values Exp(1)."""
    nnz = max(1, int(round(frac * n)))
    x = np.zeros(n)
    idx = rng.choice(n, size=nnz, replace=False)
    x[idx] = rng.exponential(1.0, size=nnz)
    return x


def random_csr(rng, m, n, density):
    """m x n CSR with each row's columns drawn uniformly without replacement
    (duplicates of a with-replacement draw removed), N(0,1) values."""
    per_row = rng.binomial(n, density, size=m)
    rows = np.repeat(np.arange(m, dtype=np.int64), per_row)
    cols = rng.integers(0, n, size=rows.size, dtype=np.int64)
    key = np.sort(rows * n + cols)
    key = key[np.concatenate([[True], key[1:] != key[:-1]])] if key.size else key
    rows, cols = key // n, key % n
    rowptr = np.zeros(m + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(np.bincount(rows, minlength=m))
    val = rng.standard_normal(cols.size)
    return rowptr.astype(np.int32), cols.astype(np.int32), val.astype(np.float32)


# ------------------------------------------------------------- problem kinds
def deconv(n_x=1000, L=100, sigma=None, support=0.05, noise=0.01, seed=BASE_SEED + 1):
    """Nonnegative deconvolution (Section 5.3): minimise ||kernel * x - b||_2
    subject to x >= 0, over variables (x, t)::

        minimise t   s.t.  x >= 0,  ||K x - b_obs||_2 <= t

    with K the full (n_x + L - 1) x n_x convolution.  Rows: n_x nonnegative
    rows (A = [-I, 0], b = 0), then one SOC of size n_x + L: head row
    (A = [0, -1], b = 0) and tail rows (A = [-K, 0], b = -b_obs).
    """
    rng = rng_for(seed)
    if sigma is None:
        sigma = L / 10.0
    kernel = gaussian_kernel(L, sigma).astype(np.float32)
    x_hat = sparse_nonneg_signal(rng, n_x, support)
    m_obs = n_x + L - 1
    b_obs = np.convolve(kernel.astype(np.float64), x_hat) + noise * rng.standard_normal(m_obs)
    A = vstack([
        hstack([scale(-1.0, eye(n_x)), zero(n_x, 1)]),
        hstack([zero(1, n_x), scale(-1.0, eye(1))]),
        hstack([scale(-1.0, conv1d(kernel, n_x)), zero(m_obs, 1)]),
    ])
    b = np.concatenate([np.zeros(n_x), [0.0], -b_obs])
    c = np.zeros(n_x + 1)
    c[-1] = 1.0
    return {"A": A, "b": b, "c": c, "cone": {"z": 0, "l": n_x, "q": [m_obs + 1]},
            "family": "deconv",
            "meta": {"n_x": n_x, "L": L, "sigma": sigma, "kernel": kernel,
                     "x_hat": x_hat, "b_obs": b_obs, "seed": seed}}


def lasso(m_d=2000, p=1000, support=0.01, noise=0.01, lam_frac=0.1, storage="fp32",
          seed=BASE_SEED + 3, data=None):
    """Lasso (Section 5.2): minimise (1/2)||D x - b||^2 + lam ||x||_1,
    lam = lam_frac * ||D^T b||_inf, over variables (x, t, w)::

        minimise w + lam 1^T t  s.t.  t - x >= 0, t + x >= 0,
                 ||(w - 1, sqrt2 (D x - b))||_2 <= w + 1

    (the SOC encodes ||D x - b||^2 <= 2 w).  D has i.i.d. N(0, 1/m_d) entries.
    """
    rng = rng_for(seed)
    if data is None:
        D = (rng.standard_normal((m_d, p)) / np.sqrt(m_d)).astype(np.float32)
    else:
        D = np.ascontiguousarray(data, dtype=np.float32)
        m_d, p = D.shape
    x_star = np.zeros(p)
    k = max(1, int(round(support * p)))
    idx = rng.choice(p, size=k, replace=False)
    x_star[idx] = rng.standard_normal(k)
    b_obs = D.astype(np.float64) @ x_star + noise * rng.standard_normal(m_d)
    lam = lam_frac * np.abs(D.astype(np.float64).T @ b_obs).max()
    r2 = np.sqrt(2.0)
    A = vstack([
        hstack([eye(p), scale(-1.0, eye(p)), zero(p, 1)]),
        hstack([scale(-1.0, eye(p)), scale(-1.0, eye(p)), zero(p, 1)]),
        hstack([zero(1, p), zero(1, p), scale(-1.0, eye(1))]),
        hstack([zero(1, p), zero(1, p), scale(-1.0, eye(1))]),
        hstack([scale(-r2, dense(D, storage)), zero(m_d, p), zero(m_d, 1)]),
    ])
    b = np.concatenate([np.zeros(2 * p), [1.0, -1.0], -r2 * b_obs])
    c = np.concatenate([np.zeros(p), lam * np.ones(p), [1.0]])
    return {"A": A, "b": b, "c": c, "cone": {"z": 0, "l": 2 * p, "q": [m_d + 2]},
            "family": "lasso",
            "meta": {"m_d": m_d, "p": p, "lam": lam, "D": D, "b_obs": b_obs,
                     "x_star": x_star, "storage": storage, "seed": seed}}


def _lasso_cone(Dtree, D_mv, D_rmv, m_d, p, rng, support, noise, lam_frac):
    """The lasso cone form of ``lasso`` around any operator D (``Dtree`` with
    FP64 products ``D_mv`` / ``D_rmv`` for the observation and lam)."""
    x_star = np.zeros(p)
    k = max(1, int(round(support * p)))
    idx = rng.choice(p, size=k, replace=False)
    x_star[idx] = rng.standard_normal(k)
    b_obs = D_mv(x_star) + noise * rng.standard_normal(m_d)
    lam = lam_frac * np.abs(D_rmv(b_obs)).max()
    r2 = np.sqrt(2.0)
    A = vstack([
        hstack([eye(p), scale(-1.0, eye(p)), zero(p, 1)]),
        hstack([scale(-1.0, eye(p)), scale(-1.0, eye(p)), zero(p, 1)]),
        hstack([zero(1, p), zero(1, p), scale(-1.0, eye(1))]),
        hstack([zero(1, p), zero(1, p), scale(-1.0, eye(1))]),
        hstack([scale(-r2, Dtree), zero(m_d, p), zero(m_d, 1)]),
    ])
    b = np.concatenate([np.zeros(2 * p), [1.0, -1.0], -r2 * b_obs])
    c = np.concatenate([np.zeros(p), lam * np.ones(p), [1.0]])
    return {"A": A, "b": b, "c": c, "cone": {"z": 0, "l": 2 * p, "q": [m_d + 2]},
            "family": "lasso", "meta": {"m_d": m_d, "p": p, "lam": lam, "b_obs": b_obs, "x_star": x_star}}


def lasso_sparse(m_d=2000, p=1000, density=0.01, support=0.01, noise=0.01, lam_frac=0.1, storage="fp32",
                 seed=BASE_SEED + 5):
    """The sparse-matrix lasso of Section 5.2: D sparse with the given
    density (the text's 1%), N(0,1) values scaled by 1/sqrt(m_d density) so
    that columns have unit expected norm as in the dense case; same cone form
    as ``lasso``."""
    rng = rng_for(seed)
    rowptr, col, val = random_csr(rng, m_d, p, density)
    val = (val / np.sqrt(m_d * density)).astype(np.float32)
    vq = val.astype(np.float64)   # the observation uses the float32 values, as in ``lasso``
    rows = np.repeat(np.arange(m_d), np.diff(rowptr))
    mv = lambda x: np.bincount(rows, weights=vq * x[col], minlength=m_d)
    rmv = lambda y: np.bincount(col, weights=vq * y[rows], minlength=p)
    out = _lasso_cone(csr(m_d, p, rowptr, col, val, storage), mv, rmv, m_d, p, rng, support, noise, lam_frac)
    out["meta"].update({"density": density, "storage": storage, "seed": seed, "operator": "csr"})
    return out


def lasso_conv(p=1000, L=None, sigma=None, support=0.01, noise=0.01, lam_frac=0.1, seed=BASE_SEED + 6):
    """The convolution lasso of Section 5.2: D x = k * x (full convolution)
    with a Gaussian kernel of length L (default p) and standard deviation
    sigma (default L/10), so m_d = p + L - 1; same cone form as ``lasso``."""
    rng = rng_for(seed)
    L = p if L is None else L
    sigma = L / 10.0 if sigma is None else sigma
    kernel = gaussian_kernel(L, sigma).astype(np.float32)
    k64 = kernel.astype(np.float64)
    m_d = p + L - 1
    mv = lambda x: np.convolve(k64, x)
    rmv = lambda y: np.correlate(y, k64, mode="valid")
    out = _lasso_cone(conv1d(kernel, p), mv, rmv, m_d, p, rng, support, noise, lam_frac)
    out["meta"].update({"L": L, "sigma": sigma, "kernel": kernel, "seed": seed, "operator": "conv1d"})
    return out


def deconv2d(h=32, w=32, kh=7, kw=7, sigma=None, support=0.05, noise=0.01, seed=BASE_SEED + 7):
    """Nonnegative 2-D deconvolution (image deblurring, the 2-D convolution
    case Section 2 motivates): minimise ||K x - b||_2 s.t. x >= 0 for an
    h x w image x (row-major) and the full 2-D convolution K with a sampled
    kh x kw Gaussian (normalised to sum 1); cone form as ``deconv``."""
    from scipy.signal import convolve2d
    rng = rng_for(seed)
    sigma = max(kh, kw) / 4.0 if sigma is None else sigma
    gy = np.exp(-((np.arange(kh) - (kh - 1) / 2.0) ** 2) / (2 * sigma * sigma))
    gx = np.exp(-((np.arange(kw) - (kw - 1) / 2.0) ** 2) / (2 * sigma * sigma))
    K = np.outer(gy, gx)
    K = (K / K.sum()).astype(np.float32)
    n_x = h * w
    x_hat = sparse_nonneg_signal(rng, n_x, support)
    Ho, Wo = h + kh - 1, w + kw - 1
    b_obs = convolve2d(x_hat.reshape(h, w), K.astype(np.float64), mode="full").ravel()
    b_obs = b_obs + noise * rng.standard_normal(Ho * Wo)
    m_obs = Ho * Wo
    A = vstack([
        hstack([scale(-1.0, eye(n_x)), zero(n_x, 1)]),
        hstack([zero(1, n_x), scale(-1.0, eye(1))]),
        hstack([scale(-1.0, conv2d(K, h, w)), zero(m_obs, 1)]),
    ])
    b = np.concatenate([np.zeros(n_x), [0.0], -b_obs])
    c = np.zeros(n_x + 1)
    c[-1] = 1.0
    return {"A": A, "b": b, "c": c, "cone": {"z": 0, "l": n_x, "q": [m_obs + 1]},
            "family": "deconv2d",
            "meta": {"h": h, "w": w, "kernel": K, "x_hat": x_hat, "b_obs": b_obs, "seed": seed}}


def lp(m_d=400, n_x=200, density=0.02, storage="fp32", seed=BASE_SEED + 4):
    """Sparse LP: minimise c^T x s.t. D x <= b, x >= 0, made feasible and
    bounded by construction (b = D x0 + slack, c = -D^T y0 with x0, slack,
    y0 >= 0).  Cone form: A = [D; -I], b = (b, 0), all rows nonnegative."""
    rng = rng_for(seed)
    rowptr, col, val = random_csr(rng, m_d, n_x, density)
    x0 = rng.uniform(0.0, 1.0, n_x)
    slack = rng.uniform(0.0, 1.0, m_d)
    y0 = rng.uniform(0.0, 1.0, m_d)
    rows = np.repeat(np.arange(m_d), np.diff(rowptr))
    Dx0 = np.bincount(rows, weights=val.astype(np.float64) * x0[col], minlength=m_d)
    DTy0 = np.bincount(col, weights=val.astype(np.float64) * y0[rows], minlength=n_x)
    b_d = Dx0 + slack
    c = -DTy0
    A = vstack([csr(m_d, n_x, rowptr, col, val, storage), scale(-1.0, eye(n_x))])
    b = np.concatenate([b_d, np.zeros(n_x)])
    return {"A": A, "b": b, "c": c, "cone": {"z": 0, "l": m_d + n_x, "q": []},
            "family": "lp",
            "meta": {"m_d": m_d, "n_x": n_x, "density": density, "seed": seed,
                     "x0": x0, "y0": y0, "storage": storage}}


def lp_batch_sizes(count=512, m_lo=200, m_hi=20000, d_lo=0.005, d_hi=0.02,
                   seed=BASE_SEED + 40):
    """Sizes of a batch of sparse LPs: m ~ U{m_lo..m_hi}, n = m // 2,
    density ~ U[d_lo, d_hi]; problem i is generated with seed + 1 + i."""
    rng = rng_for(seed)
    ms = rng.integers(m_lo, m_hi + 1, size=count)
    ds = rng.uniform(d_lo, d_hi, size=count)
    return [(int(m), int(m) // 2, float(d), seed + 1 + i) for i, (m, d) in enumerate(zip(ms, ds))]


def dense_lp(D, b_d, c, storage="fp32"):
    """min c^T x s.t. D x <= b_d, x >= 0 with a dense D (small test LPs)."""
    D = np.asarray(D, dtype=np.float32)
    m_d, n_x = D.shape
    A = vstack([dense(D, storage), scale(-1.0, eye(n_x))])
    b = np.concatenate([np.asarray(b_d, dtype=np.float64), np.zeros(n_x)])
    return {"A": A, "b": b, "c": np.asarray(c, dtype=np.float64),
            "cone": {"z": 0, "l": m_d + n_x, "q": []}, "family": "lp", "meta": {}}


def random_tiny_lp(rng, m_d, n_x, kind="feasible"):
    """Tiny dense LPs for brute-force vertex enumeration: ``feasible``
    (bounded, feasible), ``infeasible`` (a row forces sum x <= -1 with x >= 0)
    or ``unbounded`` (c has a negative entry on a column D never constrains
    upward)."""
    D = np.round(rng.uniform(-1.0, 1.0, (m_d, n_x)), 2)
    if kind == "feasible":
        D[0] = np.abs(D[0]) + 0.1           # keeps x bounded: sum_j |D0j| x_j <= b0
        b_d = np.round(rng.uniform(0.5, 2.0, m_d), 2)
        c = np.round(rng.uniform(-1.0, 1.0, n_x), 2)
    elif kind == "infeasible":
        b_d = np.round(rng.uniform(0.5, 2.0, m_d), 2)
        D[0] = 1.0
        b_d[0] = -1.0
        c = np.round(rng.uniform(-1.0, 1.0, n_x), 2)
    elif kind == "unbounded":
        D[:, 0] = -np.abs(D[:, 0]) - 0.1    # column 0 only loosens constraints
        b_d = np.round(rng.uniform(0.5, 2.0, m_d), 2)
        c = np.round(rng.uniform(-1.0, 1.0, n_x), 2)
        c[0] = -1.0
    else:
        raise ValueError(kind)
    return D, b_d, c


def mixed_cone_problem(rng, n=6, soc_sizes=(3, 4), z=1, l=3):
    """A small random feasible problem mixing all three cones: A dense random,
    s0 drawn inside K, x0 random, b = A x0 + s0, y0 inside K*, c = -A^T y0
    (so both primal and dual are feasible)."""
    m = z + l + sum(soc_sizes)
    Am = rng.standard_normal((m, n)).astype(np.float32)
    x0 = rng.standard_normal(n)
    s0 = np.zeros(m)
    y0 = np.zeros(m)
    s0[z:z + l] = rng.uniform(0.1, 1.0, l)
    y0[:z] = rng.standard_normal(z)
    y0[z:z + l] = rng.uniform(0.1, 1.0, l)
    off = z + l
    for q in soc_sizes:
        for vec in (s0, y0):
            tail = rng.standard_normal(q - 1)
            vec[off] = np.linalg.norm(tail) + rng.uniform(0.1, 1.0)
            vec[off + 1:off + q] = tail
        off += q
    b = Am.astype(np.float64) @ x0 + s0
    c = -Am.astype(np.float64).T @ y0
    return {"A": dense(Am), "b": b, "c": c,
            "cone": {"z": z, "l": l, "q": list(soc_sizes)}, "family": "mixed", "meta": {}}
