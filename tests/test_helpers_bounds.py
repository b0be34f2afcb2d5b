"""The tolerance helpers the GPU parity tests use, pinned on the CPU: the
FFT-convolution bound accepts a float32 FFT convolution (computed here with
scipy's single-precision FFT) and rejects plausible mistakes -- an output
shifted by one, a dropped tap, a wrong-sign term -- so the GPU tests that
apply it are not vacuous."""
import numpy as np
import pytest
import scipy.fft

from paper_1609_03488_b300 import synth
from tests.helpers import assert_fft_conv


def _fft_conv32(k, x, nfft=4096):
    """Overlap-save convolution in complex64 with nfft-point transforms (the
    arithmetic class of the GPU's FFT leaf)."""
    L, n = k.size, x.size
    V = nfft - L + 1
    H = scipy.fft.fft(np.concatenate([k, np.zeros(nfft - L)]).astype(np.complex64))
    z = np.concatenate([np.zeros(L - 1, np.float32), x, np.zeros(nfft, np.float32)])
    y = np.empty(n + L - 1, np.float32)
    for i0 in range(0, n + L - 1, V):
        seg = z[i0:i0 + nfft].astype(np.complex64)
        c = scipy.fft.ifft(scipy.fft.fft(seg) * H).real.astype(np.float32)
        cnt = min(V, n + L - 1 - i0)
        y[i0:i0 + cnt] = c[L - 1:L - 1 + cnt]
    return y


@pytest.mark.parametrize("kind", ["gaussian", "normal"])
def test_fft_bound_accepts_float32_fft_and_rejects_planted_mistakes(kind):
    rng = np.random.default_rng(4)
    L, n = 1000, 20000
    k = (synth.gaussian_kernel(L, 100.0) if kind == "gaussian" else rng.standard_normal(L)).astype(np.float32)
    x = rng.standard_normal(n).astype(np.float32)
    ref = np.convolve(k.astype(np.float64), x.astype(np.float64))
    y = _fft_conv32(k, x)
    assert_fft_conv(y, ref, k, x, "float32 FFT")
    # mistakes planted at the largest tap (a Gaussian's edge taps are ~1e-8 of
    # its peak: dropping one of those is below float32 resolution, no mistake)
    j = int(np.argmax(np.abs(k)))
    k_drop = k.copy()
    k_drop[j] = 0.0
    shifted_x = np.concatenate([np.zeros(j, np.float32), x, np.zeros(L - 1 - j, np.float32)])
    bad = {
        "shifted": np.roll(y, 1),
        "dropped tap": _fft_conv32(k_drop, x),
        "sign": y - 2 * k[j] * shifted_x,
    }
    for name, yb in bad.items():
        with pytest.raises(AssertionError):
            assert_fft_conv(yb, ref, k, x, name)


def test_fp32_matvec_bound_accepts_float32_sums_and_rejects_planted_mistakes():
    """The entrywise bound gamma_{k+2} (|A| |x|) of the direct kernels: a
    float32 matrix-vector product (any summation order) passes; a dropped
    column, a wrong-sign entry and a product rounded to bfloat16 fail."""
    from tests.helpers import assert_fp32_matvec
    rng = np.random.default_rng(5)
    m, n = 300, 2000
    A = rng.standard_normal((m, n)).astype(np.float32)
    x = rng.standard_normal(n).astype(np.float32)
    ref = A.astype(np.float64) @ x.astype(np.float64)
    absref = np.abs(A).astype(np.float64) @ np.abs(x).astype(np.float64)
    y = np.zeros(m, np.float32)
    for j in range(n):                       # sequential float32 sum: the worst order
        y = (y + A[:, j] * x[j]).astype(np.float32)
    assert_fp32_matvec(y, ref, absref, n, "float32 sum")
    assert_fp32_matvec(A @ x, ref, absref, n, "float32 BLAS")
    j = int(np.argmax(np.abs(x)))
    bad = {"dropped column": y - A[:, j] * x[j],
           "sign": y - 2 * A[:, j] * x[j],
           "bf16": (y.view(np.uint32) & 0xFFFF0000).view(np.float32)}
    for name, yb in bad.items():
        with pytest.raises(AssertionError):
            assert_fp32_matvec(yb, ref, absref, n, name)
