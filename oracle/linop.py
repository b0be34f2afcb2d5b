"""Structured linear operators in FP64 (test infrastructure).

Section 3.1 of the paper argues for keeping ``A`` as a composition of
structured linear operators (convolution, Kronecker products, sparse and dense
blocks) instead of a stuffed sparse matrix, and Section 4.1 derives the
adjoint of such a composition by transforming its graph.  This module gives
each node of an operator tree (format described in the input generator
module) two plain meanings:

* ``densify(op)``: the explicit float64 matrix, built entry by entry from the
  operator's definition (small problems only);
* ``apply(op, x)`` / ``apply_adjoint(op, y)``: the same map applied without
  materialising it, for sizes where the dense matrix would not fit
  (Section 5.3's point about large convolutions).

Definitions used (row-major flattening everywhere):

* conv1d, full: ``(k * x)[i] = sum_l k[l] x[i-l]``, output length n + L - 1;
  adjoint ``(K^T y)[j] = sum_l k[l] y[j+l]``.
* conv2d, full: ``Y[a, b] = sum_{p,q} K[p, q] X[a-p, b-q]``, output
  (h + kh - 1) x (w + kw - 1).
* kron: ``(A (x) B)[(i,k), (j,l)] = A[i,j] B[k,l]``.
"""
from __future__ import annotations

import numpy as np

from . import quant


# ------------------------------------------------------------------ densify
def _dense_conv1d(kernel, n):
    k = np.asarray(kernel, dtype=np.float64)
    L = k.size
    T = np.zeros((n + L - 1, n))
    for j in range(n):
        T[j:j + L, j] = k
    return T


def _dense_conv2d(kernel, h, w):
    K = np.asarray(kernel, dtype=np.float64)
    kh, kw = K.shape
    H, W = h + kh - 1, w + kw - 1
    T = np.zeros((H * W, h * w))
    for a in range(h):
        for b in range(w):
            col = a * w + b
            for p in range(kh):
                for q in range(kw):
                    T[(a + p) * W + (b + q), col] += K[p, q]
    return T


def _dense_csr(m, n, rowptr, col, val, storage):
    vals = np.asarray(val, dtype=np.float32)
    if storage == "bf16":
        vals = quant.bf16_round(vals)
    T = np.zeros((m, n))
    for i in range(m):
        for k in range(rowptr[i], rowptr[i + 1]):
            T[i, col[k]] += float(vals[k])
    return T


def densify(op):
    """Explicit float64 matrix of an operator tree node."""
    kind = op["kind"]
    if kind == "dense":
        return quant.dense_values(op["data"], op["storage"])
    if kind == "csr":
        return _dense_csr(op["m"], op["n"], op["rowptr"], op["col"], op["val"],
                          op.get("storage", "fp32"))
    if kind == "conv1d":
        return _dense_conv1d(op["kernel"], op["n"])
    if kind == "conv2d":
        return _dense_conv2d(op["kernel"], op["h"], op["w"])
    if kind == "diag":
        d = op["d"]
        return np.eye(op["n"]) if d is None else np.diag(np.asarray(d, dtype=np.float64))
    if kind == "zero":
        return np.zeros((op["m"], op["n"]))
    parts = [densify(p) for p in op.get("parts", [])]
    if kind == "scale":
        return float(op["alpha"]) * parts[0]
    if kind == "adjoint":
        return parts[0].T.copy()
    if kind == "vstack":
        return np.vstack(parts)
    if kind == "hstack":
        return np.hstack(parts)
    if kind == "blockdiag":
        T = np.zeros((op["m"], op["n"]))
        r = c = 0
        for P in parts:
            T[r:r + P.shape[0], c:c + P.shape[1]] = P
            r += P.shape[0]
            c += P.shape[1]
        return T
    if kind == "sum":
        return sum(parts[1:], parts[0].copy())
    if kind == "product":
        T = parts[0]
        for P in parts[1:]:
            T = T @ P
        return T
    if kind == "kron":
        return np.kron(parts[0], parts[1])
    raise ValueError(kind)


# ------------------------------------------------------------ matrix-free
def _leaf_matrix(op):
    # cached per storage: trees that share a leaf's data may store it differently
    cache = op.setdefault("_oracle_cache", {})
    key = ("M", op.get("storage", "fp32"))
    if key not in cache:
        if op["kind"] == "dense":
            cache[key] = quant.dense_values(op["data"], op["storage"])
        else:
            import scipy.sparse as sp
            vals = np.asarray(op["val"], dtype=np.float32)
            if op.get("storage", "fp32") == "bf16":
                vals = quant.bf16_round(vals)
            cache[key] = sp.csr_matrix((vals.astype(np.float64), op["col"], op["rowptr"]),
                                       shape=(op["m"], op["n"]))
    return cache[key]


def apply(op, x, adjoint=False):
    """``A x`` (or ``A^T x`` with ``adjoint=True``) in float64, matrix-free."""
    x = np.asarray(x, dtype=np.float64)
    kind = op["kind"]
    if kind in ("dense", "csr"):
        M = _leaf_matrix(op)
        return np.asarray(M.T @ x if adjoint else M @ x).ravel()
    if kind == "conv1d":
        k = np.asarray(op["kernel"], dtype=np.float64)
        if not adjoint:
            return np.convolve(k, x)
        # (K^T y)[j] = sum_l k[l] y[j+l]: correlation, "valid" part
        return np.correlate(x, k, mode="valid")
    if kind == "conv2d":
        from scipy.signal import convolve2d, correlate2d
        K = np.asarray(op["kernel"], dtype=np.float64)
        h, w = op["h"], op["w"]
        kh, kw = K.shape
        if not adjoint:
            return convolve2d(x.reshape(h, w), K, mode="full").ravel()
        return correlate2d(x.reshape(h + kh - 1, w + kw - 1), K, mode="valid").ravel()
    if kind == "diag":
        d = op["d"]
        return x.copy() if d is None else np.asarray(d, dtype=np.float64) * x
    if kind == "zero":
        return np.zeros(op["n"] if adjoint else op["m"])
    parts = op.get("parts", [])
    if kind == "scale":
        return float(op["alpha"]) * apply(parts[0], x, adjoint)
    if kind == "adjoint":
        return apply(parts[0], x, not adjoint)
    if kind == "vstack":
        if not adjoint:
            return np.concatenate([apply(p, x) for p in parts])
        out = np.zeros(op["n"])
        r = 0
        for p in parts:
            out += apply(p, x[r:r + p["m"]], True)
            r += p["m"]
        return out
    if kind == "hstack":
        if adjoint:
            return np.concatenate([apply(p, x, True) for p in parts])
        out = np.zeros(op["m"])
        c = 0
        for p in parts:
            out += apply(p, x[c:c + p["n"]])
            c += p["n"]
        return out
    if kind == "blockdiag":
        outs, r = [], 0
        for p in parts:
            din = p["m"] if adjoint else p["n"]
            outs.append(apply(p, x[r:r + din], adjoint))
            r += din
        return np.concatenate(outs)
    if kind == "sum":
        return sum(apply(p, x, adjoint) for p in parts)
    if kind == "product":
        seq = parts if adjoint else parts[::-1]
        v = x
        for p in seq:
            v = apply(p, v, adjoint)
        return v
    if kind == "kron":
        Aop, Bop = parts
        if not adjoint:
            X = x.reshape(Aop["n"], Bop["n"])
            T = np.stack([apply(Bop, X[j]) for j in range(Aop["n"])])       # nA x mB
            Y = np.stack([apply(Aop, T[:, k]) for k in range(Bop["m"])], 1)  # mA x mB
            return Y.ravel()
        X = x.reshape(Aop["m"], Bop["m"])
        T = np.stack([apply(Bop, X[j], True) for j in range(Aop["m"])])
        Y = np.stack([apply(Aop, T[:, k], True) for k in range(Bop["n"])], 1)
        return Y.ravel()
    raise ValueError(kind)


def shape(op):
    return op["m"], op["n"]


def nnz(op):
    """Number of stored entries if the operator were stuffed as a sparse
    matrix the way the paper's tables count them: explicit zeros of dense
    blocks are not counted, convolutions count every tap."""
    kind = op["kind"]
    if kind == "dense":
        return int(np.count_nonzero(op["data"]))
    if kind == "csr":
        return int(len(op["col"]))
    if kind == "conv1d":
        return int(np.asarray(op["kernel"]).size * op["n"])
    if kind == "diag":
        return op["n"] if op["d"] is None else int(np.count_nonzero(op["d"]))
    if kind == "zero":
        return 0
    if kind in ("scale", "adjoint"):
        return nnz(op["parts"][0])
    if kind in ("vstack", "hstack", "blockdiag", "sum"):
        return sum(nnz(p) for p in op["parts"])
    return int(np.count_nonzero(densify(op)))
