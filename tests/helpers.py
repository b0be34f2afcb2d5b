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


def assert_fft_conv(y, ref, kernel, x, what="", n_fft=4096):
    """Error bounds of a float32 overlap-save FFT convolution with n_fft-point
    transforms.  The FFT error analysis (radix-2 levels, twiddles accurate to
    u; Higham, Accuracy and Stability of Numerical Algorithms, Thm 24.2)
    bounds the 2-norm error of each transform by log2(n_fft) eta ||.||,
    eta ~ (4 sqrt2 + 1) u; a forward transform, the product with the
    spectrum (|H| <= ||h||_1) and the inverse give, per output block,
    ||err||_2 <= (2 log2(n_fft) eta + 2u) ||h||_1 ||seg||_2 with ||seg||_2 <=
    sqrt2 ||x||_2 (two overlapping segments per transform).  Asserted
    entrywise with a factor 1.5 of slack, plus a few roundings of the output;
    and the RMS error, which grows like u sqrt(log2 n_fft) on average, below
    1e-5 of ||y||."""
    lg = np.log2(n_fft)
    eta = (4 * np.sqrt(2) + 1) * U32
    blk = 1.5 * (2 * lg * eta + 2 * U32) * np.abs(np.asarray(kernel, np.float64)).sum() \
        * np.sqrt(2) * np.linalg.norm(np.asarray(x, np.float64))
    err = np.abs(np.asarray(y, dtype=np.float64) - ref)
    bound = blk + 4 * U32 * np.abs(ref)
    bad = err > bound
    assert not bad.any(), f"{what}: {bad.sum()} entries exceed the FFT bound; worst ratio {np.max(err / bound):.3g}"
    rms = np.linalg.norm(err) / max(np.linalg.norm(ref), 1e-300)
    assert rms <= 1e-5, f"{what}: relative 2-norm error {rms:.3g}"


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def fp64_residuals(prob, x, y, s):
    """pri / dual / gap of a returned point, recomputed in FP64 by the oracle."""
    from oracle import scs
    return scs.residuals(scs.Operator(prob["A"]), prob["b"], prob["c"], x, y, s)


def objective_rel_err(p, p_star):
    """|p - p*| / (1 + |p*|)."""
    return abs(p - p_star) / (1.0 + abs(p_star))


def fp32_conv_trajectory(prob, k_max, method="fft", **solve_kw):
    """The oracle's trajectory with every 1-D convolution of the iterations
    evaluated in float32 -- by scipy's single-precision FFT (method "fft") or
    by a sequential float32 direct sum over the taps ("direct"), neither of
    them this library's -- the equilibration kept exact: how far float32
    rounding of the operator alone moves the iterates.  Returns (exact,
    perturbed) oracle results."""
    import scipy.fft as sfft

    from oracle import equil, linop, scs
    kw = dict(max_iters=k_max, check_interval=10 ** 6, linsys="cg", cg_fixed_steps=3, trajectory=k_max)
    kw.update(solve_kw)
    eq_kw = kw.pop("equilibrate", None)
    eq = (equil.equilibrate(scs.Operator(prob["A"]), prob["cone"], prob["b"], prob["c"], **eq_kw)
          if eq_kw else None)
    exact = scs.solve(prob["A"], prob["b"], prob["c"], prob["cone"], equil=eq, **kw)
    plain = linop.apply

    def conv32(op, x, adjoint=False):
        if op["kind"] != "conv1d":
            return plain(op, x, adjoint)
        k = np.asarray(op["kernel"], dtype=np.float32)
        v = np.asarray(x, dtype=np.float32)
        L = k.size
        if method == "fft":
            if not adjoint:
                m = v.size + L - 1
                nf = sfft.next_fast_len(m)
                return sfft.irfft(sfft.rfft(v, nf) * sfft.rfft(k, nf), nf)[:m].astype(np.float64)
            n = v.size - L + 1
            nf = sfft.next_fast_len(v.size)
            return sfft.irfft(sfft.rfft(v, nf) * np.conj(sfft.rfft(k, nf)), nf)[:n].astype(np.float64)
        if not adjoint:
            out = np.zeros(v.size + L - 1, dtype=np.float32)
            for j in range(L):
                out[j:j + v.size] += k[j] * v
            return out.astype(np.float64)
        n = v.size - L + 1
        out = np.zeros(n, dtype=np.float32)
        for j in range(L):
            out += k[j] * v[j:j + n]
        return out.astype(np.float64)

    linop.apply = conv32
    try:
        pert = scs.solve(prob["A"], prob["b"], prob["c"], prob["cone"], equil=eq, **kw)
    finally:
        linop.apply = plain
    return exact, pert
