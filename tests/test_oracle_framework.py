"""Pins of the oracle's framework layer (Algorithm 1, Algorithm 2, Eq. 1) with the
PCZ coder plugged in, against what the paper fixes: the error bound evaluated
independently with numpy, monotone error, the equality of Alg. 2 with Alg. 1's
running sum, incremental refinement, the lossless limit, and the scalar
float-float special case of Sec. 3."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import synth_fields as S


def _err_T(x, y):
    """max |fl_T(x - y)|: Eq. 1 evaluated in the field's own precision, by numpy."""
    return float(np.max(np.abs(np.subtract(x, y, dtype=x.dtype))))


CASES = [
    # name, field, schedule
    ("gauss64_f64_delta4", lambda: S.gaussians((64, 64, 64), seed=1), "bin4", 4),
    ("pl32_f32_decade", lambda: S.powerlaw((32, 32, 32), seed=2, dtype=np.float32), "dec", 8),
    ("pl32_f64_decade", lambda: S.powerlaw((32, 32, 32), seed=2, dtype=np.float64), "dec", 8),
    ("ragged3d_f32", lambda: S.gaussians((13, 10, 7), seed=4, dtype=np.float32), "bin4", 5),
    ("ragged2d_f64", lambda: S.powerlaw((37, 22), seed=6, dtype=np.float64), "dec", 6),
    ("ragged1d_f32", lambda: S.powerlaw((203,), seed=8, dtype=np.float32), "bin4", 6),
    ("fronts24_f64", lambda: S.fronts((24, 24, 24), seed=5), "dec", 12),
]


def _tau(x, kind, n):
    r = O.value_range(x)
    return O.tau_binary(r, 4, n) if kind == "bin4" else O.tau_decade(r, n)


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def coded(request):
    _, make, kind, n = request.param
    x = make()
    tau = _tau(x, kind, n)
    return x, tau, O.Streams(x, tau, nthreads=4)


def test_eq1_bound_and_monotone_error(coded):
    x, tau, s = coded
    prev = math.inf
    for k in range(1, s.n + 1):
        err = _err_T(x, s.retrieve(k))
        assert err <= tau[k - 1], (k, err, tau[k - 1])
        assert err <= prev
        prev = err
        assert s.stats(k - 1)[O.ST_VIOL] == 0


def test_measured_error_is_computed_tolerance(coded):
    """Sec. 4.3: the computed tolerance of component i is ||x - x~_i||_inf,
    here evaluated independently by numpy on Algorithm 2's reconstruction; it
    never exceeds the prescribed tau_i, and the query on computed tolerances
    never needs more components than the query on prescribed ones."""
    x, tau, s = coded
    meas = [s.measured(i) for i in range(s.n)]
    for k in range(1, s.n + 1):
        assert meas[k - 1] == _err_T(x, s.retrieve(k)), k
        assert meas[k - 1] <= tau[k - 1]
    rng = np.random.default_rng(2)
    for t in tau[0] * 10.0 ** (-rng.uniform(0.0, 9.0, 20)):
        if t < min(meas):
            continue
        km = min(i + 1 for i in range(s.n) if meas[i] <= t)
        assert km == O.query_k(meas, t)
        assert _err_T(x, s.retrieve(km)) <= t
        if t >= tau[-1]:
            assert km <= O.query_k(tau, t)


def test_alg2_reproduces_alg1_sum(coded):
    x, tau, s = coded
    assert np.array_equal(s.retrieve(s.n), s.final_xt())


def test_incremental_equals_one_shot(coded):
    x, tau, s = coded
    for j in range(0, s.n):
        for k in range(j, s.n + 1):
            a = s.retrieve(k)
            b = s.retrieve(k, k0=j, inout=s.retrieve(j)) if j else s.retrieve(k, k0=0)
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8))


def test_subbox_is_slice_of_full(coded):
    x, tau, s = coded
    rng = np.random.default_rng(0)
    k = s.n // 2 + 1
    full = s.retrieve(k)
    for _ in range(5):
        lo = [int(rng.integers(0, d)) for d in x.shape]
        hi = [int(rng.integers(l + 1, d + 1)) for l, d in zip(lo, x.shape)]
        part = s.retrieve(k, box=(lo, hi))
        sl = tuple(slice(l, h) for l, h in zip(lo, hi))
        assert np.array_equal(part, full[sl])


def test_block_counts_and_index(coded):
    x, tau, s = coded
    for i in range(s.n):
        st = s.stats(i)
        assert st[O.ST_ZERO] + st[O.ST_CODED] + st[O.ST_RAW] == s.nbricks
        cw = s.chunk_word(i)
        bl = s.brick_len(i).astype(np.int64)
        words = 0
        for c in range(s.nchunks):
            assert cw[c] == words  # every chunk starts on its own 64-bit word
            words += (int(bl[32 * c:32 * c + 32].sum()) + 63) // 64
        assert words == len(s.payload(i))


def test_packed_bits_equal_per_brick_bits(coded):
    x, tau, s = coded
    rng = np.random.default_rng(1)
    for b in rng.integers(0, s.nbricks, size=6):
        b = int(b)
        bits, nbits, xt, st = O.code_brick(x, tau, b)
        for i in range(s.n):
            bl = s.brick_len(i).astype(np.int64)
            c = b // 32
            start = int(s.chunk_word(i)[c]) * 64 + int(bl[32 * c:b].sum())
            pl = s.payload(i)
            got = "".join(str((int(pl[(start + t) >> 6]) >> ((start + t) & 63)) & 1) for t in range(int(bl[b])))
            assert got == O.bits_to_str(bits[i], int(nbits[i]))


@pytest.mark.parametrize("dtype,n", [(np.float64, 14), (np.float32, 8)])
def test_lossless_limit(dtype, n):
    # values in [6, 14]: every nonzero residual is at least one ulp of such a
    # value, so a last tolerance below that ulp forces x~ == x bit for bit
    # (Sec. 5.1.3: enough components make the lossy coder lossless)
    x = S.powerlaw((12, 10, 9), seed=21, dtype=np.float64)
    x = (10.0 + 4.0 * x / np.abs(x).max()).astype(dtype)
    tau = O.tau_binary(O.value_range(x), 4, n)
    ulp = float(np.spacing(dtype(4.0)))
    assert tau[-1] < ulp
    s = O.Streams(x, tau)
    assert np.array_equal(s.retrieve(n).view(np.uint8), x.view(np.uint8))
    # the computed tolerance reaches 0 exactly where x~ first equals x
    meas = [s.measured(i) for i in range(n)]
    k0 = next(i + 1 for i in range(n) if meas[i] == 0.0)
    assert np.array_equal(s.retrieve(k0).view(np.uint8), x.view(np.uint8))
    assert not np.array_equal(s.retrieve(k0 - 1), x)
    assert all(m == 0.0 for m in meas[k0 - 1:])


def test_zero_field_is_all_zero_blocks():
    x = np.zeros((9, 8, 7))
    s = O.Streams(x, [1.0, 0.5])
    for i in range(2):
        assert s.stats(i)[O.ST_ZERO] == s.nbricks
        assert (s.brick_len(i) == 2).all()
    assert not s.retrieve(2).any()


def test_rejects_bad_input():
    x = np.ones((4, 4, 4))
    with pytest.raises(ValueError):
        O.Streams(x, [1.0, 1.0])  # not strictly decreasing
    with pytest.raises(ValueError):
        O.Streams(x, [1.0, 0.0])
    with pytest.raises(ValueError):
        O.Streams(x, [-1.0])
    y = x.copy()
    y[1, 2, 3] = np.nan
    with pytest.raises(ValueError):
        O.Streams(y, [1.0])  # NaN and infinities are not handled (Sec. 6.1)
    y[1, 2, 3] = np.inf
    with pytest.raises(ValueError):
        O.Streams(y, [1.0])


def test_query_k():
    tau = [1.0, 0.1, 0.01]
    assert O.query_k(tau, 5.0) == 1  # looser than tau_1: one component at least
    assert O.query_k(tau, 1.0) == 1  # ties select i
    assert O.query_k(tau, 0.5) == 2
    assert O.query_k(tau, 0.1) == 2
    assert O.query_k(tau, 0.01) == 3
    assert O.query_k(tau, 0.009) == -1  # unreachable


def test_scalar_float_float_special_case():
    # Sec. 3: with C o D = rounding to float32, Algorithm 1 on a double is the
    # float-float expansion: x_1 = fl32(x), x_2 = fl32(x - x_1), ...
    third = 1.0 / 3.0
    comps = O.scalar_fl32([third, 1.0 + 2.0 ** -30, math.pi], 4)
    # 1/3 in float32 is 0x3EAAAAAB (11184811 * 2^-25)
    assert np.float32(comps[0, 0]).view(np.uint32) == 0x3EAAAAAB
    assert Fraction(comps[0, 0]) == Fraction(11184811, 2 ** 25)
    # the second component is the exact double residual rounded to float32
    r1 = Fraction(third) - Fraction(comps[0, 0])
    assert comps[1, 0] == float(np.float32(float(r1)))
    # two components carry about 48 bits: |x - (x_1 + x_2)| <= 2^-48 |x|
    assert abs(Fraction(third) - Fraction(comps[0, 0]) - Fraction(comps[1, 0])) <= Fraction(third) * 2 ** -48
    # a double with 31 significant bits splits exactly into 1 and 2^-30
    assert list(comps[:, 1]) == [1.0, 2.0 ** -30, 0.0, 0.0]
    # pi: three float components reproduce the double exactly (53 <= 3 * 24)
    s = 0.0
    for i in range(4):
        s = s + comps[i, 2]
    assert s == math.pi
