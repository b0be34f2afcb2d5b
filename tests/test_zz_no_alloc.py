"""The allocation-free entry point cf_op_apply_static, for callers that may
not allocate GPU memory (their framework's allocator owns the device memory,
or a cudaMalloc/cudaFree in their loop would stall the GPU).

It must give the same y = A x / A^T x as the allocating entry point
cf_op_apply, on two calls in a row, with an unrelated operator's scratch
left in the shared static array between them.  Calls go on torch's current
stream (the binding's default), so they are ordered after the torch kernels
that fill their inputs and outputs.  This file is collected last on
purpose."""
import numpy as np
import pytest

from oracle import linop
from paper_1609_03488_b300 import synth
from tests.helpers import assert_fp32_matvec

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


@pytest.mark.parametrize("storage", ["fp32", "bf16", "fp8"])
def test_static_apply_matches_allocating_apply(B, ctx, storage):
    import torch
    rng = np.random.default_rng(17)
    m, n = 3000, 1200
    D = rng.standard_normal((m, n)).astype(np.float32)
    tree = synth.lasso(m_d=m, p=n, seed=5, storage=storage, data=D)["A"]   # dense leaf inside a tree
    op = B.build_operator(ctx, tree)
    assert op.workspace_bytes(adjoint=True) > 0        # the adjoint really uses scratch
    for call in range(2):                               # two calls in a row
        yv = rng.standard_normal(op.m).astype(np.float32)
        xv = rng.standard_normal(op.n).astype(np.float32)
        want_t = op.apply(yv, adjoint=True)             # existing, allocating entry point
        want = op.apply(xv)
        yd = torch.from_numpy(yv).cuda()
        xd = torch.from_numpy(xv).cuda()
        out_t = torch.full((op.n,), float("nan"), device="cuda")
        out = torch.full((op.m,), float("nan"), device="cuda")
        op.apply_static(yd, out_t, adjoint=True)
        op.apply_static(xd, out)
        torch.cuda.synchronize()
        got_t, got = out_t.cpu().numpy(), out.cpu().numpy()
        np.testing.assert_array_equal(got_t, want_t)    # same kernels, same order: bitwise
        np.testing.assert_array_equal(got, want)
        if call == 0:
            # leave unrelated values in the shared array before the second
            # call: a product whose intermediate is larger than the dense
            # adjoint's partial sums
            k = 300_000
            other = B.operator_compose(ctx, "product", [
                B.cf_op_dense(ctx, rng.standard_normal((8, k)).astype(np.float32), "fp32"),
                B.cf_op_diag(ctx, k, rng.random(k).astype(np.float32))])
            assert other.workspace_bytes() > op.workspace_bytes(adjoint=True)
            xo = torch.from_numpy(rng.standard_normal(k).astype(np.float32)).cuda()
            yo = torch.empty(8, device="cuda")
            other.apply_static(xo, yo)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(yo.cpu().numpy(), other.apply(xo.cpu().numpy()))
        # and within the float32 bound of the FP64 oracle
        ref = linop.apply(tree, yv.astype(np.float64), adjoint=True)
        absT = np.abs(linop.densify(tree))
        assert_fp32_matvec(got_t, ref, absT.T @ np.abs(yv.astype(np.float64)), m + 2, "static adjoint")


def test_static_apply_accumulate_and_alpha(B, ctx):
    import torch
    rng = np.random.default_rng(3)
    D = rng.standard_normal((500, 300)).astype(np.float32)
    op = B.cf_op_dense(ctx, D, "fp32")
    y = rng.standard_normal(500).astype(np.float32)
    base = rng.standard_normal(300).astype(np.float32)
    want = base.astype(np.float64) - 2.0 * (D.T.astype(np.float64) @ y)
    out = torch.from_numpy(base.copy()).cuda()
    op.apply_static(torch.from_numpy(y).cuda(), out, adjoint=True, alpha=-2.0, accumulate=True)
    torch.cuda.synchronize()
    bound = np.abs(base) + 2.0 * (np.abs(D.T) @ np.abs(y))
    assert_fp32_matvec(out.cpu().numpy(), want, bound, 500 + 3, "static accumulate")


def test_static_apply_rejects_oversized_scratch(B, ctx):
    import torch
    # a product with a 2.2M-long inner dimension needs two 2.2M-float
    # intermediates: 17.6 MB, more than the 16 MiB static array
    k = 2_200_000
    op = B.operator_compose(ctx, "product", [B.cf_op_zero(ctx, 5, k), B.cf_op_diag(ctx, k)])
    assert op.workspace_bytes() > (16 << 20)
    x = torch.ones(k, device="cuda")
    y = torch.empty(5, device="cuda")
    with pytest.raises(B.CfError) as e:
        op.apply_static(x, y)
    assert e.value.code == B.CF_E_INVALID
    assert "static array" in str(e.value)
