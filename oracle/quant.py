"""Reduced-precision operand formats, written from the formats' definitions
(test infrastructure; see the package docstring).

The paper runs its operators in the framework's default precision; the BF16
and FP8 operand storage modes are this library's precision axis, where the
quantised operand *defines* the problem instance: every entry is the exact
real number its code denotes (times the row scale for FP8), and the oracle
solves that instance in FP64.

* bfloat16: 1 sign, 8 exponent, 7 mantissa bits; float32 -> bfloat16 rounds to
  nearest, ties to even, on the 16 dropped bits.
* FP8 E4M3 (the "FN" variant: no infinities, max finite 448, one NaN pattern):
  exponent bias 7, subnormal quantum 2^-9; float32 -> e4m3 rounds to nearest,
  ties to even, and saturates finite values to +-448.
* per-row scale: ``s_i = max_j |a_ij| / 448`` in float32 (``s_i = 1`` for an
  all-zero row); codes ``q_ij = e4m3(a_ij / s_i)`` with the division in
  float32; the represented entry is ``q_ij * s_i``.
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0


def bf16_round(a):
    """float32 array -> float32 array holding the nearest bfloat16 values
    (ties to even).  NaN stays NaN."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    bits = a.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16) << 16
    out = rounded.astype(np.uint32).view(np.float32).copy()
    nan = np.isnan(a)
    out[nan] = np.nan
    return out


def _round_half_even(v):
    return np.round(v)          # numpy rounds halves to even


def e4m3_value(a):
    """float32 array -> float64 array of the e4m3 values it rounds to
    (nearest, ties to even, saturating to +-448)."""
    a = np.asarray(a, dtype=np.float32).astype(np.float64)
    sgn = np.sign(a)
    mag = np.abs(a)
    out = np.zeros_like(mag)
    nz = mag > 0
    # exponent of the binade, clamped to the smallest normal exponent (-6):
    # below it the quantum stays 2^-9 (subnormals).
    e = np.floor(np.log2(np.where(nz, mag, 1.0)))
    e = np.maximum(e, -6.0)
    # log2 can be off by one ulp at exact powers of two; fix the binade.
    e = np.where(np.ldexp(1.0, e.astype(int)) > mag, e - 1, e)
    e = np.where(np.ldexp(1.0, (e + 1).astype(int)) <= mag, e + 1, e)
    e = np.maximum(e, -6.0)
    quantum = np.ldexp(1.0, (e - 3).astype(int))
    q = _round_half_even(mag / quantum) * quantum
    q = np.minimum(q, E4M3_MAX)
    out[nz] = q[nz]
    res = sgn * out
    res[np.isnan(a)] = np.nan
    return res


def e4m3_code(v):
    """e4m3 values (exactly representable, as produced by ``e4m3_value``) ->
    uint8 codes (sign bit 7, exponent bits 6..3, mantissa bits 2..0)."""
    v = np.asarray(v, dtype=np.float64)
    sign = (np.signbit(v)).astype(np.uint8) << 7
    mag = np.abs(v)
    code = np.zeros(v.shape, dtype=np.uint8)
    nz = mag > 0
    e = np.floor(np.log2(np.where(nz, mag, 1.0)))
    sub = nz & (e < -6)
    # subnormal: mag = m * 2^-9
    code[sub] = np.round(mag[sub] / 2.0 ** -9).astype(np.uint8)
    nrm = nz & ~sub
    en = e[nrm].astype(int)
    man = np.round((mag[nrm] / np.ldexp(1.0, en) - 1.0) * 8).astype(int)
    code[nrm] = ((en + 7) << 3 | man).astype(np.uint8)
    code |= sign
    code[np.isnan(v)] = 0x7F
    return code


def fp8_rowwise(a):
    """Per-row-scaled e4m3 quantisation of a float32 matrix.

    Returns ``(codes uint8 m x n, scales float32 m, dequant float64 m x n)``
    where ``dequant[i, j] = value(codes[i, j]) * scales[i]`` exactly."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    amax = np.abs(a).max(axis=1).astype(np.float32)
    s = (amax / np.float32(E4M3_MAX)).astype(np.float32)
    s = np.where(amax > 0, s, np.float32(1.0)).astype(np.float32)
    ratio = (a / s[:, None]).astype(np.float32)       # float32 division
    vals = e4m3_value(ratio)
    codes = e4m3_code(vals)
    deq = vals * s.astype(np.float64)[:, None]
    return codes, s, deq


def dense_values(data, storage):
    """The exact entries (float64) of a dense operand stored as ``storage``."""
    data = np.ascontiguousarray(data, dtype=np.float32)
    if storage == "fp32":
        return data.astype(np.float64)
    if storage == "bf16":
        return bf16_round(data).astype(np.float64)
    if storage == "fp8":
        return fp8_rowwise(data)[2]
    raise ValueError(storage)
