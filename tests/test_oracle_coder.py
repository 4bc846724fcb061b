"""Pins of the oracle's block coder (the project-defined PCZ coder R4..R13)
against things other than the oracle itself: closed forms, exhaustive and
brute-force round trips, hand-built streams, numpy/math library routines and
exact rational arithmetic (fractions)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# ---------------------------------------------------------------- lifting (R7)


@pytest.mark.parametrize("P", [32, 64])
def test_lift4_exhaustive_roundtrip(P):
    # every 4-vector with entries in [-6, 6]: the integer lifting is exactly invertible
    r = range(-6, 7)
    for a in r:
        for b in r:
            for c in r:
                for d in r:
                    v = [a, b, c, d]
                    assert list(O.lift_inv4(O.lift_fwd4(v, P), P)) == v


def test_lift4_linear_ramp_has_no_detail():
    # a linear ramp (a, a+t, a+2t, a+3t) leaves only the mean and the slope
    rng = np.random.default_rng(7)
    for _ in range(2000):
        a, t = (int(z) for z in rng.integers(-2**40, 2**40, size=2))
        out = O.lift_fwd4([a, a + t, a + 2 * t, a + 3 * t], 64)
        assert out[2] == 0 and out[3] == 0
        assert out[1] == 2 * t  # coarse slope of the two pair means


def test_lift4_constant_is_dc_only():
    for c in (-5, 0, 3, 2**50):
        assert list(O.lift_fwd4([c] * 4, 64)) == [c, 0, 0, 0]


@pytest.mark.parametrize("d", [1, 2, 3])
def test_affine_block_has_only_dc_and_slopes(d):
    # an affine brick a + t1*i + t2*j + t3*l keeps at most d+1 nonzero coefficients:
    # the DC at position 0 and one slope term per axis (positions 1, 4, 16)
    rng = np.random.default_rng(11)
    N = 4 ** d
    for _ in range(200):
        a = int(rng.integers(-2**30, 2**30))
        t = [int(z) for z in rng.integers(-2**20, 2**20, size=3)]
        v = []
        for pos in range(N):
            i, j, l = pos & 3, (pos >> 2) & 3, pos >> 4
            v.append(a + t[0] * i + t[1] * j + t[2] * l)
        c = O.lift_fwd_block(v, d, 64)
        nz = {int(p) for p in np.nonzero(c)[0]}
        assert nz <= {1: {0, 1}, 2: {0, 1, 4}, 3: {0, 1, 4, 16}}[d]
        assert list(O.lift_inv_block(c, d, 64)) == v


@pytest.mark.parametrize("d,P", [(1, 32), (2, 32), (3, 32), (1, 64), (2, 64), (3, 64)])
def test_block_roundtrip_and_headroom(d, P):
    # random bricks with |q| < 2^(P-2-2d) round-trip exactly and stay below 2^(P-2)
    rng = np.random.default_rng(100 + d + P)
    N = 4 ** d
    M = 2 ** (P - 2 - 2 * d) - 1
    for _ in range(300):
        v = [int(z) for z in rng.integers(-M, M + 1, size=N)]
        c = O.lift_fwd_block(v, d, P)
        assert max(abs(int(z)) for z in c) < 2 ** (P - 2)
        assert list(O.lift_inv_block(c, d, P)) == v


@pytest.mark.parametrize("d", [1, 2, 3])
def test_forward_growth_bound_is_attained(d):
    # the separable sign pattern s(i)s(j)s(l) with s = (+,-,-,+) reaches the
    # stated L-inf growth of exactly 4^d, the headroom G = 2d bits
    M = 2 ** 20
    s = [1, -1, -1, 1]
    N = 4 ** d
    v = []
    for pos in range(N):
        i, j, l = pos & 3, (pos >> 2) & 3, pos >> 4
        v.append(M * s[i] * (s[j] if d > 1 else 1) * (s[l] if d > 2 else 1))
    c = O.lift_fwd_block(v, d, 64)
    assert max(abs(int(z)) for z in c) == 4 ** d * M
    rng = np.random.default_rng(5)
    for _ in range(500):
        v = [int(M * z) for z in rng.choice([-1, 1], size=N)]
        assert max(abs(int(z)) for z in O.lift_fwd_block(v, d, 64)) <= 4 ** d * M


@pytest.mark.parametrize("d", [1, 2, 3])
def test_inverse_gain_matches_guard(d):
    # the inverse's L-inf gain (max row sum of |inverse|, measured on large
    # impulses) is 2.75^d; the guard planes c_d are the smallest c with
    # 2^c > (2/3) * 2.75^d: 1, 3, 4
    N = 4 ** d
    S = 2 ** 30
    cols = []
    for k in range(N):
        v = [0] * N
        v[k] = S
        cols.append(np.array(O.lift_inv_block(v, d, 64), dtype=np.float64) / S)
    A = np.stack(cols, axis=1)
    gain = np.abs(A).sum(axis=1).max()
    assert abs(gain - 2.75 ** d) < 1e-6
    c = {1: 1, 2: 3, 3: 4}[d]
    assert 2 ** (c - 1) <= (2 / 3) * gain < 2 ** c


def test_perm_is_sequency_order():
    for d in (1, 2, 3):
        N = 4 ** d
        p = list(O.perm(d))
        assert sorted(p) == list(range(N))
        keys = [((pos & 3) + ((pos >> 2) & 3) + (pos >> 4), pos) for pos in p]
        assert keys == sorted(keys)
    assert list(O.perm(1)) == [0, 1, 2, 3]
    # 2D by hand: sequency 0: (0,0); 1: (1,0),(0,1); 2: (2,0),(1,1),(0,2); ...
    assert list(O.perm(2)[:6]) == [0, 1, 4, 2, 5, 8]


# -------------------------------------------------------------- negabinary (R9)


@pytest.mark.parametrize("P", [32, 64])
def test_negabinary_closed_form(P):
    for q in range(-2**15, 2**15, 7):
        u = O.nb_fwd(q, P)
        assert 0 <= u < 2 ** P
        assert sum(((u >> b) & 1) * (-2) ** b for b in range(P)) == q
        assert O.nb_inv(u, P) == q
    assert O.nb_fwd(1, P) == 1 and O.nb_fwd(-1, P) == 3 and O.nb_fwd(2, P) == 6 and O.nb_fwd(-2, P) == 2


@pytest.mark.parametrize("P", [32, 64])
def test_negabinary_extremes(P):
    # the whole range |q| < 2^(P-2) the transform can produce is representable
    for q in (2 ** (P - 2) - 1, -(2 ** (P - 2) - 1), 2 ** (P - 3), -(2 ** (P - 3))):
        u = O.nb_fwd(q, P)
        assert sum(((u >> b) & 1) * (-2) ** b for b in range(P)) == q
        assert O.nb_inv(u, P) == q


# ---------------------------------------------------- bit-plane coding (R11)


def _golden_streams():
    rows = []
    with open(os.path.join(GOLDEN, "bitplane_streams.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, bits, _why = (s.strip() for s in line.split("|"))
            N, P, pmin, us = head.split()
            u = [int(z, 2) for z in us.split(",")]
            rows.append((int(N), int(P), int(pmin), u, bits))
    return rows


@pytest.mark.parametrize("N,P,pmin,u,bits", _golden_streams())
def test_hand_built_streams(N, P, pmin, u, bits):
    words, nb = O.encode_planes(u, N, P, pmin)
    assert O.bits_to_str(words, nb) == bits
    w, n = O.str_to_bits(bits)
    dec, used = O.decode_planes(w, n, N, P, pmin)
    keep = ~((1 << pmin) - 1)
    assert used == n
    assert [int(z) for z in dec] == [z & keep for z in u]


def _all_vectors(N, P):
    import itertools
    return itertools.product(range(2 ** P), repeat=N)


@pytest.mark.parametrize("N,P", [(1, 6), (2, 6), (3, 4), (4, 3)])
def test_bitplane_bruteforce_roundtrip(N, P):
    # every coefficient vector, every lowest plane: decode(encode(u)) is u with
    # the planes below pmin cleared, and decoding reads exactly what was written
    rng = np.random.default_rng(N * 100 + P)
    for u in _all_vectors(N, P):
        pmin = int(rng.integers(0, P + 1))
        words, nb = O.encode_planes(list(u), N, P, pmin)
        # trailing garbage after the block must not be read
        garbage = np.concatenate([words, rng.integers(0, 2**63, size=2, dtype=np.uint64)])
        w2 = garbage.copy()
        if nb % 64:
            w2[nb // 64] |= np.uint64(rng.integers(0, 2**63)) << np.uint64(nb % 64)
        dec, used = O.decode_planes(w2, nb + 100, N, P, pmin)
        assert used == nb
        keep = ~((1 << pmin) - 1)
        assert [int(z) for z in dec] == [z & keep for z in u]


def test_bitplane_random_wide():
    rng = np.random.default_rng(3)
    for _ in range(3000):
        N = int(rng.choice([4, 16, 64]))
        P = int(rng.choice([32, 64]))
        top = int(rng.integers(1, P + 1))
        u = [int(z) for z in rng.integers(0, 2 ** min(top, 63), size=N, dtype=np.uint64)]
        pmin = int(rng.integers(0, P + 1))
        words, nb = O.encode_planes(u, N, P, pmin, maxbits=P * (2 * N + 1) + 64)
        dec, used = O.decode_planes(words, nb, N, P, pmin)
        assert used == nb
        keep = (2 ** 64 - 1) ^ ((1 << pmin) - 1)
        assert [int(z) for z in dec] == [z & keep for z in u]


def test_bitplane_rejects_truncated():
    words, nb = O.encode_planes([0b1010, 0b0101, 0b1010, 0b0101], 4, 4, 0)
    for cut in range(nb):
        _, used = O.decode_planes(words, cut, 4, 4, 0)
        assert used == -1


# ------------------------------------------------- alignment and scaling (R6, R13)


def test_block_emax_matches_frexp():
    rng = np.random.default_rng(9)
    for _ in range(500):
        e = rng.standard_normal(64) * 10.0 ** rng.integers(-30, 30)
        e[rng.integers(0, 64, size=5)] = 0.0
        want = max(math.frexp(float(v))[1] for v in e if v != 0)
        assert O.block_emax(e, np.float64) == max(want, -1021)
    assert O.block_emax([0.0, 5e-324], np.float64) == -1021  # subnormal: floor at the smallest normal
    assert O.block_emax([0.0, 1e-45], np.float32) == -125
    assert O.block_emax([1.0, -0.75], np.float64) == 1
    assert O.block_emax([3.4e38], np.float32) == 128


def test_quantize_is_exact_floor():
    rng = np.random.default_rng(4)
    for _ in range(2000):
        e = float(rng.standard_normal() * 10.0 ** rng.integers(-300, 300))
        emax = math.frexp(e)[1] + int(rng.integers(0, 4))
        s = 56 - emax
        want = math.floor(abs(Fraction(e)) * Fraction(2) ** s)
        want = -want if e < 0 else want
        assert O.quantize(e, s) == want
        assert abs(want) < 2 ** 56
    assert O.quantize(5e-324, 1077) == 8
    assert O.quantize(-1.5, 1) == -3 and O.quantize(-1.75, 1) == -3


def _is_rn(v, exact: Fraction, ftype):
    """v is the ftype value nearest to exact, ties to even (checked by definition)."""
    if math.isinf(v):
        # RN overflows exactly from the midpoint of the largest finite value and 2^emax
        big = Fraction(float(np.finfo(ftype).max))
        top = Fraction(2) ** (128 if ftype == np.float32 else 1024)
        return abs(exact) >= (big + top) / 2 and (v > 0) == (exact > 0)
    fv = ftype(v)
    if float(fv) != v:
        return False
    # for rounding, the neighbour past the largest finite value is 2^emax
    top = Fraction(2) ** (128 if ftype == np.float32 else 1024)

    def frac(z):
        return Fraction(z) if math.isfinite(z) else (top if z > 0 else -top)

    dn = frac(float(np.nextafter(fv, ftype(-np.inf))))
    up = frac(float(np.nextafter(fv, ftype(np.inf))))
    dv = abs(Fraction(v) - exact)
    if dv > abs(dn - exact) or dv > abs(up - exact):
        return False
    if dv == abs(dn - exact) or dv == abs(up - exact):
        bits = fv.view(np.uint32 if ftype == np.float32 else np.uint64)
        return (int(bits) & 1) == 0
    return True


@pytest.mark.parametrize("ftype", [np.float32, np.float64])
def test_dequantize_rounds_to_nearest_even(ftype):
    rng = np.random.default_rng(12)
    emin = -149 if ftype == np.float32 else -1074
    emax = 128 if ftype == np.float32 else 1024
    for _ in range(3000):
        q = int(rng.integers(-2**62, 2**62)) >> int(rng.integers(0, 62))
        if q == 0:
            continue
        s = int(rng.integers(-(emax - 40), -emin + 70))
        v = O.dequantize(q, s, ftype)
        assert _is_rn(v, Fraction(q) * Fraction(2) ** (-s), ftype), (q, s, v)
    assert O.dequantize(3, 1, ftype) == 1.5
    assert O.dequantize(0, 7, ftype) == 0.0


def test_dequantize_subnormal_single_rounding():
    # q*2^-s = (2.5 + 2^-60) units of the smallest subnormal: one correct
    # rounding gives 3 units; rounding q to 53 bits first drops the 2^-60,
    # leaves an exact tie and then rounds to the even 2 units
    q = 5 * 2**59 + 1
    s = 1074 + 60
    v = O.dequantize(q, s, np.float64)
    assert _is_rn(v, Fraction(q) * Fraction(2) ** (-s), np.float64)
    assert v == 3 * 5e-324
    assert math.ldexp(float(q), -s) == 2 * 5e-324  # the double-rounded value differs
    assert O.dequantize(-q, s, np.float64) == -3 * 5e-324


def test_dequantize_overflow_is_inf():
    assert O.dequantize(2**60, -1024 + 60 - 64 - 2, np.float64) == math.inf
    assert O.dequantize(-(2**40), -200, np.float32) == -math.inf


def test_floor_log2():
    for e in range(-1020, 1020, 37):
        t = math.ldexp(1.0, e)
        assert O.floor_log2(t) == e
        assert O.floor_log2(t * 1.999) == e
        assert O.floor_log2(math.nextafter(t, 0)) == e - 1
    assert O.floor_log2(5e-324) == -1074
    assert O.floor_log2(3 * 5e-324) == -1073
    assert O.floor_log2(math.ldexp(1.0, -1060)) == -1060


# ------------------------------------------------------------- padding (R4)


@pytest.mark.parametrize("shape", [(5,), (7,), (6, 9), (5, 3), (5, 6, 7), (1, 1, 3), (9, 4, 5)])
def test_gather_is_edge_replication(shape):
    rng = np.random.default_rng(len(shape))
    x = rng.standard_normal(shape)
    nd = len(shape)
    nb = [(s + 3) // 4 for s in shape]
    padded = np.pad(x, [(0, 4 * n - s) for n, s in zip(nb, shape)], mode="edge")
    b = 0
    for bz in range(nb[0] if nd == 3 else 1):
        for by in range(nb[-2] if nd >= 2 else 1):
            for bx in range(nb[-1]):
                got = O.gather_brick(x, b)
                if nd == 1:
                    want = padded[4 * bx:4 * bx + 4]
                elif nd == 2:
                    want = padded[4 * by:4 * by + 4, 4 * bx:4 * bx + 4]
                else:
                    want = padded[4 * bz:4 * bz + 4, 4 * by:4 * by + 4, 4 * bx:4 * bx + 4]
                assert np.array_equal(got, want.reshape(-1))
                b += 1
