"""Shared test utilities: tolerances derived from float32 arithmetic and
FP64 checks of a returned solution through the oracle."""
import numpy as np

U32 = 2.0 ** -24   # unit roundoff of float32


def assert_fp32_matvec(y, ref, absref, k, what=""):
    """Rigorous bound for a float32 sum of at most k products computed in
    any order: |y - ref| <= gamma_{k+2} * (|A| |x|), gamma_j = j u / (1 - j u)."""
    j = k + 2
    gamma = j * U32 / (1 - j * U32)
    err = np.abs(np.asarray(y, dtype=np.float64) - ref)
    bound = gamma * absref + 1e-30
    bad = err > bound
    assert not bad.any(), (f"{what}: {bad.sum()} of {bad.size} entries exceed the float32 bound; "
                           f"worst ratio {np.max(err / bound):.3g}")


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def fp64_residuals(prob, x, y, s):
    """pri / dual / gap of a returned point, recomputed in FP64 by the oracle."""
    from oracle import scs
    return scs.residuals(scs.Operator(prob["A"]), prob["b"], prob["c"], x, y, s)


def objective_rel_err(p, p_star):
    """|p - p*| / (1 + |p*|)."""
    return abs(p - p_star) / (1.0 + abs(p_star))
