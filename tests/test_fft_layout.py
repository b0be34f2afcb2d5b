"""Host checks of the FFT convolution kernel's shared-memory addressing.

The transform buffer pads one slot per 16 complex values (pad(e) = e + e // 16)
so that the innermost stage's stride-16 accesses fall on distinct banks.  The
kernel replaces pad(position) by pad(base) + a constant offset in three
places; these identities must hold for every thread of both transform sizes.
"""
import pytest


def pad(e):
    return e + (e >> 4)


@pytest.mark.parametrize("N", [2048, 4096])
def test_padded_offsets_are_constant_per_stage(N):
    T = N // 16            # threads per pair
    G = N // 16            # second-stage group length
    S = G // 16            # second-stage stride
    LS = 4 if N == 4096 else 3
    for t in range(T):
        # first forward / last inverse stage: positions t + T q
        for q in range(16):
            assert pad(t + T * q) == pad(t) + (T + T // 16) * q
        # second stage: positions base + r S
        base = G * (t >> LS) + (t & (S - 1))
        for r in range(16):
            off = 17 * r if S == 16 else 8 * r + (r >> 1)
            assert pad(base + r * S) == pad(base) + off
        # innermost stage: 16 contiguous positions 16 t + r
        for r in range(16):
            assert pad(16 * t + r) == 17 * t + r


@pytest.mark.parametrize("N", [2048, 4096])
def test_every_position_has_one_slot(N):
    T, G = N // 16, N // 16
    S = G // 16
    LS = 4 if N == 4096 else 3
    slots = set()
    for t in range(T):
        base = G * (t >> LS) + (t & (S - 1))
        for r in range(16):
            slots.add(pad(base + r * S))
    assert len(slots) == N
    assert max(slots) < N + N // 16
