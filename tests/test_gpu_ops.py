"""GPU parity of the operator kernels (Section 3.1 structured operators;
adjoints per Section 4.1) against the FP64 oracle, through the C ABI.

Float32 results are held to the rigorous bound of a float32 sum of k
products, |y - y*| <= gamma_{k+2} (|A| |x|); stored BF16/FP8 operands must
match the oracle's quantiser bit for bit.  1-D convolutions evaluated by
overlap-save FFTs are held to the FFT's error bound instead
(tests.helpers.assert_fft_conv)."""
import numpy as np
import pytest

from oracle import linop, quant
from paper_1609_03488_b300 import synth
from tests.helpers import assert_fft_conv, assert_fp32_matvec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1609_03488_b300 import build
    build.build()
    from paper_1609_03488_b300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    return B.Context(0)


def _abs_tree(node):
    """The same tree with every leaf's entries replaced by their absolute
    values (|A| for the float32 error bound)."""
    k = node["kind"]
    out = dict(node)
    if k == "dense":
        out["data"] = np.abs(node["data"])
        if node["storage"] != "fp32":      # |stored value|: quantise first
            out["data"] = np.abs(quant.dense_values(node["data"], node["storage"])).astype(np.float32)
            out["storage"] = "fp32"
    elif k == "csr":
        v = np.asarray(node["val"], np.float32)
        if node.get("storage", "fp32") == "bf16":
            v = quant.bf16_round(v)
        out["val"], out["storage"] = np.abs(v), "fp32"
    elif k in ("conv1d", "conv2d"):
        out["kernel"] = np.abs(node["kernel"])
    elif k == "diag":
        out["d"] = None if node["d"] is None else np.abs(node["d"])
    elif k == "scale":
        out["alpha"] = abs(node["alpha"])
    if "parts" in node:
        out["parts"] = [_abs_tree(p) for p in node["parts"]]
    out.pop("_oracle_cache", None)
    return out


def _check(B, ctx, tree, k_fwd, k_adj, seed=0, what=""):
    rng = np.random.default_rng(seed)
    op = B.build_operator(ctx, tree)
    assert (op.m, op.n) == (tree["m"], tree["n"])
    x = rng.standard_normal(tree["n"]).astype(np.float32)
    y = rng.standard_normal(tree["m"]).astype(np.float32)
    absT = _abs_tree(tree)
    ref = linop.apply(tree, x.astype(np.float64))
    bound = linop.apply(absT, np.abs(x).astype(np.float64))
    assert_fp32_matvec(op.apply(x), ref, bound, k_fwd, what + " forward")
    ref = linop.apply(tree, y.astype(np.float64), adjoint=True)
    bound = linop.apply(absT, np.abs(y).astype(np.float64), adjoint=True)
    assert_fp32_matvec(op.apply(y, adjoint=True), ref, bound, k_adj, what + " adjoint")


@pytest.mark.parametrize("n,L", [(1, 1), (5, 3), (3, 7), (1000, 100), (2049, 17), (3000, 1000),
                                 (5000, 2500), (70001, 1000)])
def test_conv1d(B, ctx, n, L):
    rng = np.random.default_rng(n + L)
    k = rng.standard_normal(L).astype(np.float32)
    _check(B, ctx, synth.conv1d(k, n, method="direct"), L, L, what=f"conv1d n={n} L={L}")


def _check_fft(B, ctx, k, n, method="fft", seed=0, what=""):
    rng = np.random.default_rng(seed)
    tree = synth.conv1d(k, n, method=method)
    op = B.build_operator(ctx, tree)
    x = rng.standard_normal(n).astype(np.float32)
    y = rng.standard_normal(n + k.size - 1).astype(np.float32)
    assert_fft_conv(op.apply(x), linop.apply(tree, x.astype(np.float64)), k, x, what + " forward")
    assert_fft_conv(op.apply(y, adjoint=True), linop.apply(tree, y.astype(np.float64), adjoint=True), k, y,
                    what + " adjoint")
    return op, x, y


# one output, a single pair, ragged tails around the 2V-output pairs (V =
# N + 1 - Lp: 4096-point transforms for kernels over 1024 padded taps or
# outputs enough to fill the GPU, else 2048-point), the largest kernel (2048
# taps, V = 2049), the largest 2048-point kernel (1024 taps, V = 1025) and the
# next, tiny kernels, and 2e6 outputs on 4096-point transforms
@pytest.mark.parametrize("n,L", [(1, 1000), (5, 16), (1000, 100), (3000, 1000), (6177, 1000), (6178, 1000),
                                 (20000, 2048), (70001, 1000), (4099, 257), (100, 3),
                                 (1083, 1000), (1084, 1000), (2082, 1000), (5000, 1024), (5000, 1025),
                                 (2_000_000, 1000)])
def test_conv1d_fft(B, ctx, n, L):
    rng = np.random.default_rng(7 * n + L)
    k = rng.standard_normal(L).astype(np.float32)
    _check_fft(B, ctx, k, n, what=f"conv1d fft n={n} L={L}")


def test_conv1d_method_selection(B, ctx):
    """auto = FFT for 256..2048 padded taps (bitwise), direct below; the FFT
    method refuses longer kernels."""
    rng = np.random.default_rng(5)
    x = rng.standard_normal(9000).astype(np.float32)
    for L, auto_is in ((240, "direct"), (241, "fft"), (2048, "fft"), (2049, "direct")):
        k = rng.standard_normal(L).astype(np.float32)
        a = B.build_operator(ctx, synth.conv1d(k, 9000, method="auto")).apply(x)
        b = B.build_operator(ctx, synth.conv1d(k, 9000, method=auto_is)).apply(x)
        np.testing.assert_array_equal(a, b)
    with pytest.raises(B.CfError) as e:
        B.build_operator(ctx, synth.conv1d(rng.standard_normal(2049).astype(np.float32), 100, method="fft"))
    assert e.value.code == B.CF_E_INVALID


def test_conv1d_fft_adjoint_identity_and_accumulate(B, ctx):
    rng = np.random.default_rng(6)
    k = rng.standard_normal(700).astype(np.float32)
    op, x, y = _check_fft(B, ctx, k, 15000, what="conv1d fft n=15000")
    lhs = float(op.apply(x).astype(np.float64) @ y)
    rhs = float(x.astype(np.float64) @ op.apply(y, adjoint=True))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(op.apply(x)) * np.linalg.norm(y)
    import torch
    dev = torch.device("cuda", 0)
    xd = torch.from_numpy(x).to(dev)
    yd = torch.from_numpy(y).to(dev)
    ws = torch.empty(max(op.workspace_bytes(False) // 4, 1), device=dev)
    op.apply_async(xd, yd, alpha=-0.5, accumulate=True, workspace=ws)   # y - 0.5 A x
    torch.cuda.synchronize()
    want = y.astype(np.float64) - 0.5 * linop.apply(synth.conv1d(k, 15000), x.astype(np.float64))
    assert_fft_conv(yd.cpu().numpy(), want, 0.5 * k, x, "accumulate")


def test_deconv_tree_with_fft_convolution(B, ctx):
    """The cone-form deconvolution operator with an FFT (and a direct)
    convolution leaf: the -I blocks' rows are exact and the convolution rows
    meet the FFT bound, both directions."""
    prob = synth.deconv(n_x=5000, L=300, seed=12)
    k = prob["meta"]["kernel"]
    n_x = 5000
    rng = np.random.default_rng(13)
    for method in ("fft", "direct"):
        tree = synth.with_conv_method(prob["A"], method)
        op = B.build_operator(ctx, tree)
        x = rng.standard_normal(tree["n"]).astype(np.float32)
        y = rng.standard_normal(tree["m"]).astype(np.float32)
        fx, fy = op.apply(x), op.apply(y, adjoint=True)
        np.testing.assert_array_equal(fx[:n_x], -x[:n_x])
        assert fx[n_x] == -x[n_x]
        ref = linop.apply(tree, x.astype(np.float64))
        assert_fft_conv(fx[n_x + 1:], ref[n_x + 1:], k, x[:n_x], f"deconv tree {method} forward")
        ref = linop.apply(tree, y.astype(np.float64), adjoint=True)
        assert fy[n_x] == -y[n_x]
        assert_fft_conv(fy[:n_x], ref[:n_x], k, y[n_x + 1:], f"deconv tree {method} adjoint")


@pytest.mark.parametrize("method", ["direct", "fft"])
def test_conv1d_full_size_large_deconvolution(B, ctx, method):
    """The n = 1e6, L = 1000 (sigma = 100) Gaussian operator of the large
    deconvolution workload, both directions, every output, both methods."""
    k = synth.gaussian_kernel(1000, 100.0).astype(np.float32)
    if method == "direct":
        _check(B, ctx, synth.conv1d(k, 1_000_000, method="direct"), 1000, 1000, what="conv1d 1e6")
    else:
        _check_fft(B, ctx, k, 1_000_000, what="conv1d fft 1e6")


@pytest.mark.parametrize("h,w,kh,kw", [(1, 5, 2, 3), (30, 40, 5, 7), (64, 50, 31, 17), (17, 19, 64, 1)])
def test_conv2d(B, ctx, h, w, kh, kw):
    rng = np.random.default_rng(h * w + kh)
    K = rng.standard_normal((kh, kw)).astype(np.float32)
    _check(B, ctx, synth.conv2d(K, h, w), kh * kw, kh * kw, what=f"conv2d {h}x{w} k{kh}x{kw}")


@pytest.mark.parametrize("storage", ["fp32", "bf16", "fp8"])
@pytest.mark.parametrize("m,n", [(1, 1), (37, 53), (1000, 777), (3000, 2500)])
def test_dense(B, ctx, storage, m, n):
    rng = np.random.default_rng(m * 7 + n)
    D = (rng.standard_normal((m, n)) * rng.uniform(0.01, 10, (m, 1))).astype(np.float32)
    tree = synth.dense(D, storage)
    _check(B, ctx, tree, n, m, what=f"dense {storage} {m}x{n}")


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_dense_stored_codes_bit_exact(B, ctx, storage):
    rng = np.random.default_rng(5)
    D = (rng.standard_normal((300, 517)) * 10.0 ** rng.uniform(-3, 3, (300, 1))).astype(np.float32)
    D[7] = 0.0
    D[11, :5] = [448.0, -464.0, 1e-9, 3 * 2.0 ** -10, 0.0]
    op = B.cf_op_dense(ctx, D, storage)
    codes, scales = op.dense_stored(B.PREC[storage])
    if storage == "bf16":
        want = quant.bf16_round(D).view(np.uint32) >> 16
        np.testing.assert_array_equal(codes.astype(np.uint32), want)
    else:
        wc, ws, _ = quant.fp8_rowwise(D)
        np.testing.assert_array_equal(scales, ws)
        np.testing.assert_array_equal(codes, wc)


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
@pytest.mark.parametrize("m,n,dens", [(1, 1, 1.0), (300, 200, 0.05), (2000, 1000, 0.02), (50, 4000, 0.3)])
def test_csr(B, ctx, storage, m, n, dens):
    rng = np.random.default_rng(m + n)
    rp, col, val = synth.random_csr(rng, m, n, dens)
    tree = synth.csr(m, n, rp, col, val, storage)
    kmax = max(int(np.diff(rp).max(initial=0)), 1)
    kcol = max(int(np.bincount(col, minlength=n).max(initial=0)), 1)
    _check(B, ctx, tree, kmax, kcol, what=f"csr {storage} {m}x{n}")


def test_csr_empty_rows_and_columns(B, ctx):
    rp = np.array([0, 0, 2, 2], np.int32)
    col = np.array([0, 2], np.int32)
    val = np.array([1.5, -2.0], np.float32)
    _check(B, ctx, synth.csr(3, 4, rp, col, val), 2, 2, what="csr empty rows")


def test_diag_zero_scale(B, ctx):
    rng = np.random.default_rng(3)
    d = rng.standard_normal(1001).astype(np.float32)
    _check(B, ctx, synth.scale(-2.5, synth.diag(1001, d)), 1, 1, what="diag")
    _check(B, ctx, synth.eye(17), 1, 1, what="identity")
    tree = synth.vstack([synth.zero(3, 5), synth.eye(5)])
    _check(B, ctx, tree, 1, 1, what="zero")


def test_kron(B, ctx):
    rng = np.random.default_rng(8)
    A = rng.standard_normal((7, 5)).astype(np.float32)
    Bm = rng.standard_normal((6, 4)).astype(np.float32)
    tree = synth.kron(synth.dense(A), synth.dense(Bm))
    # two chained float32 products: k = 4 + 5 terms bounds each output
    _check(B, ctx, tree, 4 * 5 + 9, 7 * 6 + 13, what="kron")
    # the named entry point is the same operator, bit for bit
    op1 = B.build_operator(ctx, tree)
    op2 = B.cf_op_kron(ctx, B.cf_op_dense(ctx, A), B.cf_op_dense(ctx, Bm))
    x = rng.standard_normal(20).astype(np.float32)
    y = rng.standard_normal(42).astype(np.float32)
    np.testing.assert_array_equal(op1.apply(x), op2.apply(x))
    np.testing.assert_array_equal(op1.apply(y, adjoint=True), op2.apply(y, adjoint=True))
    with pytest.raises(B.CfError):
        B.cf_op_kron(ctx, B.cf_op_dense(ctx, A), B.cf_op_diag(ctx, 4))


def test_random_composition_tree(B, ctx):
    from tests.test_oracle_linop import _rand_tree
    rng = np.random.default_rng(4)
    tree = _rand_tree(rng)
    op = B.build_operator(ctx, tree)
    T = linop.densify(tree)
    for s in range(3):
        x = rng.standard_normal(tree["n"]).astype(np.float32)
        y = rng.standard_normal(tree["m"]).astype(np.float32)
        np.testing.assert_allclose(op.apply(x), T @ x.astype(float), rtol=2e-5, atol=2e-5 * np.abs(T).sum(1).max())
        np.testing.assert_allclose(op.apply(y, adjoint=True), T.T @ y.astype(float), rtol=2e-5,
                                   atol=2e-5 * np.abs(T).sum(0).max())


def test_deconv_and_lasso_trees(B, ctx):
    p = synth.deconv(n_x=700, L=64, seed=9)
    _check(B, ctx, p["A"], 64, 66, what="deconv A")
    q = synth.lasso(m_d=300, p=128, seed=9, storage="bf16")
    _check(B, ctx, q["A"], 128, 302, what="lasso A")


def test_device_pointers(B, ctx):
    import torch
    rng = np.random.default_rng(1)
    D = rng.standard_normal((64, 48)).astype(np.float32)
    op = B.cf_op_dense(ctx, torch.from_numpy(D).cuda(), "fp32")
    x = torch.from_numpy(rng.standard_normal(48).astype(np.float32)).cuda()
    y = torch.empty(64, dtype=torch.float32, device="cuda")
    op.apply(x, out=y)
    torch.cuda.synchronize()
    ref = D.astype(float) @ x.cpu().numpy().astype(float)
    assert_fp32_matvec(y.cpu().numpy(), ref, np.abs(D) @ np.abs(x.cpu().numpy()), 48, "device ptrs")


def test_measured_fma_rates_are_plausible(B, ctx):
    """cf_measure_fma_rate, the measured denominator of the ALU rooflines:
    float32 within [0.5, 1.05] of SMs x 128 lanes x 2 flop x the maximum SM
    clock (2032 MHz on B300), float64 positive and well below float32."""
    fp32 = ctx.fma_rate(False)
    fp64 = ctx.fma_rate(True)
    nominal = ctx.sm_count * 128 * 2 * 2032e6
    assert 0.5 * nominal <= fp32 <= 1.05 * nominal, (fp32, nominal)
    assert 0 < fp64 < 0.5 * fp32, (fp64, fp32)
