"""The identity behind float64 retrieval's 32-bit decoding of narrow brick
pairs, checked with the oracle's own integer transform (R7) and negabinary
map (R9).

A pair whose coded planes lie in [lo, lo + 16) with lo >= 6 and no digit
above plane 58 is decoded by the retrieval kernel in 32-bit integers in units
of 2^(lo - 6): negabinary digits v from plane lo stand for
((v ^ M) - M) * 2^lo with M = NBM >> lo, and each pass of the inverse lifting
turns multiples of 2^a into multiples of 2^(a - 2), so every shift is exact
and the three passes end on integers.  Here the 64-bit inverse transform of
the coefficients must equal the 32-bit (wrapping) inverse transform of the
scaled ones, shifted back, and the scaled values must stay far inside int32.
Random digits and the extreme patterns (every digit of one sign's planes
set) are both tried."""
import numpy as np
import pytest

import oracle as O

NBM64 = 0xAAAAAAAAAAAAAAAA


def _to_int32(u):
    u &= 0xFFFFFFFF
    return u - (1 << 32) if u >> 31 else u


def _digits(rng, span, mode):
    if span <= 0:
        return [0] * 64
    if mode == 0:
        return [int(v) for v in rng.integers(0, 1 << span, size=64)]
    even = sum(1 << k for k in range(0, span, 2))  # the largest positive value
    odd = sum(1 << k for k in range(1, span, 2))   # the most negative one
    if mode == 1:
        return [even] * 64
    return [even if rng.random() < 0.5 else odd for _ in range(64)]


@pytest.mark.parametrize("max_span", [16, 21])
def test_scaled_inverse_transform_is_exact(max_span):
    rng = np.random.default_rng(max_span)
    for trial in range(240):
        lo = int(rng.integers(6, 59))
        hi = int(rng.integers(lo - 1, min(lo + max_span - 1, 58) + 1))
        v = _digits(rng, hi - lo + 1, trial % 3)
        c64 = [O.nb_inv(d << lo, 64) for d in v]
        want = O.lift_inv_block(c64, 3, 64)
        m = (NBM64 >> lo) & 0xFFFFFFFF
        c32 = [_to_int32(((d ^ m) - m) << 6) for d in v]
        got = O.lift_inv_block(c32, 3, 32)
        assert np.array_equal(got.astype(object) * (1 << (lo - 6)), want.astype(object)), (lo, hi)
        # the bound of the kernel's comment: |value| < 2^(hi - lo + 10.8)
        assert int(np.abs(got).max()) < 2.0 ** (hi - lo + 10.8)
