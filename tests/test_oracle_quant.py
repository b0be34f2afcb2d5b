"""Pins for the oracle's reduced-precision operand formats.

Each format is checked against values fixed by its definition (hand-decoded
codes, ties-to-even cases) and against an independent implementation of the
same cast (PyTorch's CPU dtype conversions)."""
import numpy as np
import pytest
import torch

from oracle import quant


def _decode_e4m3(code):
    s = -1.0 if code & 0x80 else 1.0
    e = (code >> 3) & 0xF
    mnt = code & 0x7
    if e == 0:
        return s * mnt * 2.0 ** -9
    return s * (1.0 + mnt / 8.0) * 2.0 ** (e - 7)


def test_bf16_matches_torch_cast():
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10.0 ** rng.integers(-30, 30, 20000),
                        np.array([1.0, -2.5, 3.0e38, 1e-40, 0.0, -0.0], dtype=np.float32)]).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(quant.bf16_round(a), ref)


def test_bf16_ties_to_even():
    # 1 + 2^-8 lies halfway between bf16 neighbours 1 and 1 + 2^-7: rounds to 1 (even).
    a = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8], dtype=np.float32)
    np.testing.assert_array_equal(quant.bf16_round(a), np.array([1.0, 1.0 + 2 * 2.0 ** -7], dtype=np.float32))


def test_e4m3_fixed_values():
    cases = {1.0: 0x38, 448.0: 0x7E, 2.0 ** -9: 0x01, 2.0 ** -6: 0x08, -1.5: 0xBC,
             0.875 * 2.0 ** -6: 0x07, 240.0: 0x77}
    for val, code in cases.items():
        v = quant.e4m3_value(np.array([val], dtype=np.float32))
        assert v[0] == val
        assert quant.e4m3_code(v)[0] == code
        assert _decode_e4m3(code) == val


def test_e4m3_ties_and_saturation():
    a = np.array([1.0625, 1.1875, 500.0, -1e6, 2.0 ** -10, 3 * 2.0 ** -10, 464.0], dtype=np.float32)
    expect = np.array([1.0, 1.25, 448.0, -448.0, 0.0, 2 * 2.0 ** -9, 448.0])
    np.testing.assert_array_equal(quant.e4m3_value(a), expect)


def test_e4m3_matches_torch_cast_in_range():
    rng = np.random.default_rng(1)
    a = (rng.standard_normal(50000) * 10.0 ** rng.uniform(-4, 2.6, 50000)).astype(np.float32)
    a = a[np.abs(a) <= 448.0]
    ref = torch.from_numpy(a).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(quant.e4m3_value(a), ref)
    codes = quant.e4m3_code(quant.e4m3_value(a))
    ref_codes = torch.from_numpy(a).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    np.testing.assert_array_equal(codes, ref_codes)


def test_every_code_roundtrips():
    for code in range(256):
        if code & 0x7F == 0x7F:
            continue  # NaN
        val = _decode_e4m3(code)
        v = quant.e4m3_value(np.array([val], dtype=np.float32))
        assert v[0] == val
        got = quant.e4m3_code(v)[0]
        if val == 0.0:
            assert got & 0x7F == 0
        else:
            assert got == code


@pytest.mark.parametrize("shape", [(7, 33), (64, 1000)])
def test_fp8_rowwise_error_bound(shape):
    rng = np.random.default_rng(2)
    a = rng.standard_normal(shape).astype(np.float32)
    a[0] = 0.0
    codes, s, deq = quant.fp8_rowwise(a)
    assert s[0] == 1.0 and np.all(deq[0] == 0.0)
    # largest entry of each row maps to +-448 exactly
    for i in range(1, shape[0]):
        j = np.argmax(np.abs(a[i]))
        assert abs(deq[i, j] / s[i]) == 448.0
    # relative rounding error of a normal e4m3 value is at most 2^-4
    big = np.abs(a) >= 2.0 ** -6 * s[:, None] * 1.01
    rel = np.abs(deq - a)[big] / np.abs(a)[big]
    assert rel.max() <= 2.0 ** -4 * 1.0001
