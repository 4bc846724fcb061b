"""Pins of the oracle's enforcement of Eq. 1 in floating point (Sec. 4.3): the
verification of every block on the sum it will produce, escalation (a lower
coded plane when the check fails, rule R13), RAW storage of the residual when
no coded precision meets tau (R13; raw storage on expansion, Sec. 5.1.1), the
choice between a passing CODED block and RAW (R14), and the counting of the
violations that floating point can leave (Sec. 4.3).

What they are pinned against, besides the oracle itself:
  * a RAW block written out by hand (tests/golden/raw_block.txt);
  * the IEEE bit patterns of the residual (struct/numpy views);
  * Eq. 1 evaluated with numpy in the field's type;
  * a re-composition of Algorithm 1 and the block coder's decisions from the
    unit steps that tests/test_oracle_coder.py pins one by one (exponent
    against frexp, quantisation against exact rationals, lifting by brute
    force, negabinary by its closed form, bit planes by hand-built streams,
    dequantisation against the definition of round-to-nearest-even).
The inputs that reach escalation and the R14 tie are rare, so they were found
by a seeded search (tests/golden/find_enforcement_cases.py) and are stored.
"""
import os

import numpy as np
import pytest

import oracle as O
import synth_fields as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MODE_ZERO, MODE_CODED, MODE_RAW = 0, 1, 2


# ------------------------------------------------------------------ the model


def _lsb(v: int, width: int) -> str:
    """A field written least significant bit first (R12)."""
    return "".join(str((v >> b) & 1) for b in range(width))


def _params(dt, d):
    P = 32 if dt == np.float32 else 64
    ebits, ebias = (8, 126) if dt == np.float32 else (11, 1022)
    return P, P - 2 - 2 * d, {1: 1, 2: 3, 3: 4}[d], ebits, ebias


def _eq1_ok(x, xt, xi, tau, dt):
    """Eq. 1 on the sum the block will produce, in the field's type (R13)."""
    with np.errstate(over="ignore", invalid="ignore"):
        r = np.abs(x.astype(dt) - (xt.astype(dt) + xi.astype(dt)))
    return bool(np.all(r.astype(np.float64) <= tau))


def model_block(x, xt, tau, dt, d):
    """What rules R5, R6, R10, R13 and R14 make of one full brick, composed from
    the separately pinned unit steps.  Returns (mode, esc, bits, x_i)."""
    P, Q, c, ebits, ebias = _params(dt, d)
    N = 4 ** d
    with np.errstate(over="ignore", invalid="ignore"):
        e = (x.astype(dt) - xt.astype(dt)).astype(dt)
    if np.all(np.abs(e.astype(np.float64)) <= tau):  # R5
        return MODE_ZERO, 0, "00", np.zeros(N, dtype=dt)
    raw_bits = "01" + "".join(_lsb(int(b), P) for b in e.view(np.uint32 if dt == np.float32 else np.uint64))
    if not np.all(np.isfinite(e)):
        return MODE_RAW, 0, raw_bits, e
    emax = O.block_emax(e.astype(np.float64), dt)  # R6
    s = Q - emax
    q = [O.quantize(float(v), s) for v in e]
    coef = O.lift_fwd_block(q, d, P)  # R7
    perm = O.perm(d)  # R8
    u = [O.nb_fwd(int(coef[perm[r]]), P) for r in range(N)]  # R9
    L = O.floor_log2(tau)
    passed = False
    for esc in range(8):  # R10, R13
        p = min(max(L + s - c - esc, 0), P)
        keep = ((1 << P) - 1) & ~((1 << p) - 1)
        qt = [0] * N
        for r in range(N):
            qt[perm[r]] = O.nb_inv(u[r] & keep, P)
        back = O.lift_inv_block(qt, d, P)
        xi = np.array([O.dequantize(int(v), s, dt) for v in back], dtype=np.float64).astype(dt)
        if _eq1_ok(x, xt, xi, tau, dt):
            passed = True
            break
        if esc == 7 or p == 0:
            break
    if passed:
        words, nb = O.encode_planes(u, N, P, p, maxbits=N * P * 3)
        len_coded, len_raw = 2 + 3 + ebits + nb, 2 + N * P
        if not (len_coded > len_raw and _eq1_ok(x, xt, e, tau, dt)):  # R14
            bits = _lsb(MODE_CODED, 2) + _lsb(esc, 3) + _lsb(emax + ebias, ebits) + O.bits_to_str(words, nb)
            return MODE_CODED, esc, bits, xi
    return MODE_RAW, 0, raw_bits, e


def model_brick(x, taus, dt):
    """Algorithm 1 on one full brick with the model coder: x~ <- 0; per component
    e = x - x~, y_i = C(e, tau_i), x~ <- x~ + D(y_i), sums in the field's type."""
    d = x.ndim
    xf = x.reshape(-1).astype(dt)
    xt = np.zeros(xf.size, dtype=dt)
    out = []
    for tau in taus:
        mode, esc, bits, xi = model_block(xf, xt, tau, dt, d)
        with np.errstate(over="ignore"):
            xt = (xt + xi.astype(dt)).astype(dt)
        out.append((mode, esc, bits))
    return out, xt


def oracle_strings(x, taus):
    bits, nbits, xt, st = O.code_brick(x, taus, 0, maxwords=256)
    return [O.bits_to_str(bits[i], nbits[i]) for i in range(len(taus))], xt, st


def _field(dtname, hexes):
    dt = np.float32 if dtname == "f32" else np.float64
    ints = np.array([int(h, 16) for h in hexes.split(",")], dtype=np.uint32 if dt == np.float32 else np.uint64)
    return ints.view(dt), dt


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [[p.strip() for p in ln.split("|")] for ln in f if ln.strip() and not ln.startswith("#")]


# ------------------------------------------------------------- RAW storage


def test_raw_block_written_by_hand():
    (dtname, hexes, tau_hex, want), = _rows("raw_block.txt")
    x, dt = _field(dtname, hexes)
    tau = float.fromhex(tau_hex)
    got, xt, st = oracle_strings(x, [tau])
    assert got[0] == want.replace(" ", "")
    assert list(st[0]) == [0, 0, 1, 0, 0]  # one RAW block, no violation
    # D(y_1) is the residual (= x, since x~_0 = 0) bit for bit
    bits, nbits, _, _ = O.code_brick(x, [tau], 0)
    back = O.decode_brick(dt, 1, [tau], 1, bits, nbits).astype(dt)
    assert np.array_equal(back.view(np.uint32), x.view(np.uint32))
    assert model_brick(x, [tau], dt)[0][0][2] == got[0]


def test_raw_every_brick_of_float32_noise():
    # uniform noise in (-1, 1) at tau = 2^-26: lanes below 1/2 lose bits to the
    # block exponent even with every plane coded, so bricks are stored RAW and
    # the first reconstruction is x itself
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, size=(16, 16, 16)).astype(np.float32)
    s = O.Streams(x, [2.0 ** -26])
    st = s.stats(0)
    assert st[O.ST_RAW] == s.nbricks and st[O.ST_VIOL] == 0
    assert np.array_equal(s.retrieve(1).view(np.uint32), x.view(np.uint32))
    assert s.measured(0) == 0.0


# ------------------------------------------------------------- R14


def test_r14_longer_coded_block_is_stored_raw():
    # four float32 values of one binade, in no smooth order: every plane coded
    # reproduces them exactly (the quantisation is exact), but that takes more
    # than the 2 + 4*32 bits of RAW storage
    x = np.array([1.9, 1.1, 1.7, 1.3], dtype=np.float32)
    tau = 2.0 ** -40
    got, _, st = oracle_strings(x, [tau])
    assert st[0, O.ST_RAW] == 1
    assert got[0] == "01" + "".join(_lsb(int(b), 32) for b in x.view(np.uint32))
    # the CODED alternative passes Eq. 1 and is longer
    P, Q, c, ebits, _ = _params(np.float32, 1)
    emax = O.block_emax(x.astype(np.float64), np.float32)
    q = [O.quantize(float(v), Q - emax) for v in x]
    assert O.lift_inv_block(O.lift_fwd_block(q, 1, P), 1, P).tolist() == q
    assert [O.dequantize(v, Q - emax, np.float32) for v in q] == [float(v) for v in x]
    coef = O.lift_fwd_block(q, 1, P)
    u = [O.nb_fwd(int(coef[r]), P) for r in O.perm(1)]
    _, nb = O.encode_planes(u, 4, P, 0)
    assert 2 + 3 + ebits + nb > 2 + 4 * P
    assert model_brick(x, [tau], np.float32)[0][0][0] == MODE_RAW


@pytest.mark.parametrize("row", _rows("r14_ties_1d.txt"), ids=lambda r: r[0] + ":" + r[1][:8])
def test_r14_tie_keeps_coded(row):
    x, dt = _field(row[0], row[1])
    tau = float.fromhex(row[2])
    P = 32 if dt == np.float32 else 64
    got, _, st = oracle_strings(x, [tau])
    assert len(got[0]) == 2 + 4 * P and got[0][:2] == _lsb(MODE_CODED, 2)
    assert st[0, O.ST_CODED] == 1
    # RAW would meet tau as well (it reproduces x), so only the tie rule keeps CODED
    assert _eq1_ok(x, np.zeros(4, dt), x, tau, dt)
    assert model_brick(x, [tau], dt)[0][0][2] == got[0]


# ------------------------------------------------------------- escalation


@pytest.mark.parametrize("row", _rows("escalation_1d.txt"), ids=lambda r: r[0] + ":" + r[1][:8])
def test_escalation_lowers_the_plane_by_one_per_round(row):
    x, dt = _field(row[0], row[1])
    taus = [float.fromhex(t) for t in row[2].split()]
    got, xt, st = oracle_strings(x, taus)
    assert st[1, O.ST_CODED] == 1 and st[1, O.ST_ESC] >= 1
    modes, xt_model = model_brick(x, taus, dt)
    mode, esc, bits = modes[1]
    assert (mode, esc) == (MODE_CODED, int(st[1, O.ST_ESC]))
    assert bits == got[1]  # header esc field and the planes down to p0 - esc
    assert [m[2] for m in modes] == got
    assert np.array_equal(xt.astype(dt), xt_model)
    assert np.all(np.abs(x.astype(np.float64) - xt) <= taus[1])


def _near_top(dt, frac, shape=(16, 16, 16), seed=7):
    """magnitudes in [frac, 1] of the largest finite value, signs of a k^-5/3 field
    (one-signed for float64, so that the range max - min stays finite)."""
    base = S.powerlaw(shape, seed=seed, dtype=np.float64)
    base = base / np.abs(base).max()
    top = float(np.finfo(dt).max)
    mag = (frac + (1 - frac) * np.abs(base)) * top
    x = (mag if dt == np.float64 else np.sign(base) * mag).astype(dt)
    return x


@pytest.mark.parametrize("dt,frac,kind", [(np.float32, 0.9999, "bin"), (np.float32, 0.999, "dec"),
                                          (np.float64, 0.9, "bin"), (np.float64, 0.99, "dec")])
def test_escalation_and_raw_at_the_top_of_the_range(dt, frac, kind):
    # reconstructions of values near the largest finite value round to infinity
    # at the first precision tried, so the coder escalates (and stores some
    # blocks RAW); every decision is the rules' and Eq. 1 holds
    x = _near_top(dt, frac)
    r = O.value_range(x)
    taus = O.tau_binary(r, 4, 6) if kind == "bin" else O.tau_decade(r, 6)
    s = O.Streams(x, taus)
    assert sum(s.stats(i)[O.ST_ESC] for i in range(6)) > 0
    for k in range(1, 7):
        xk = s.retrieve(k)
        assert np.all(np.isfinite(xk))
        err = np.abs(x.astype(np.float64) - xk.astype(np.float64))
        assert int(np.sum(err > taus[k - 1])) == s.stats(k - 1)[O.ST_VIOL] == 0
    # brick by brick, the oracle's strings are the rules' (bricks with escalation first)
    checked = 0
    for b in range(s.nbricks):
        bits, nbits, _, st = O.code_brick(x, taus[:2], b, maxwords=256)
        if st[:, O.ST_ESC].sum() == 0 and st[:, O.ST_RAW].sum() == 0 and b % 16:
            continue
        bz, by, bx = b // 16, (b // 4) % 4, b % 4
        brick = x[4 * bz:4 * bz + 4, 4 * by:4 * by + 4, 4 * bx:4 * bx + 4]
        modes, _ = model_brick(np.ascontiguousarray(brick), taus[:2], dt)
        assert [m[2] for m in modes] == [O.bits_to_str(bits[i], nbits[i]) for i in range(2)], b
        checked += 1
    assert checked >= 4


# ------------------------------------------------------------- violations


@pytest.mark.parametrize("dt,shape", [(np.float32, (4096,)), (np.float64, (4096,)),
                                      (np.float32, (16, 16, 16)), (np.float64, (16, 16, 16))])
def test_violations_left_by_floating_point_are_counted(dt, shape):
    # a coarse first component leaves x~_1 far from small values of x (more than
    # a factor 2 away), so fl(x - x~_1) is inexact and even RAW storage of the
    # residual cannot meet a tau below its rounding error (Sec. 4.3).  The
    # counters must equal the violations of Eq. 1 counted with numpy.
    rng = np.random.default_rng(3)
    x = (rng.normal(size=shape) * 2.0 ** rng.uniform(-8, 0, size=shape)).astype(dt)
    mant = 24 if dt == np.float32 else 53
    taus = [0.25, 2.0 ** -(mant + 6)]
    s = O.Streams(x, taus)
    assert s.stats(1)[O.ST_RAW] > 0
    viol = 0
    for k in (1, 2):
        xk = s.retrieve(k)
        err = np.abs(x - xk).astype(np.float64)  # |fl_T(x - x~_k)|
        assert int(np.sum(err > taus[k - 1])) == s.stats(k - 1)[O.ST_VIOL]
        assert s.measured(k - 1) == float(err.max())
        viol += s.stats(k - 1)[O.ST_VIOL]
    assert viol > 0
    if x.ndim == 3:  # the rules' decisions on a few bricks, RAW ones included
        for b in (0, 5, 17, 63):
            bz, by, bx = b // 16, (b // 4) % 4, b % 4
            brick = np.ascontiguousarray(x[4 * bz:4 * bz + 4, 4 * by:4 * by + 4, 4 * bx:4 * bx + 4])
            bits, nbits, _, _ = O.code_brick(x, taus, b, maxwords=256)
            modes, _ = model_brick(brick, taus, dt)
            assert [m[2] for m in modes] == [O.bits_to_str(bits[i], nbits[i]) for i in range(2)]


# ------------------------------------------------------------- random bricks


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_block_decisions_follow_the_rules(d, dt):
    # random full bricks, 3 components at tolerances from coarse down to the ulp
    # level: every component's string is the one the rules compose
    rng = np.random.default_rng(40 + d + (dt == np.float64))
    mant = 24 if dt == np.float32 else 53
    modes_seen = set()
    for _ in range(60 if d < 3 else 12):
        x = (rng.normal(size=(4,) * d) * 2.0 ** rng.uniform(-6, 0, size=(4,) * d)).astype(dt)
        top = float(rng.uniform(-4, 0))
        taus = sorted((2.0 ** (top - float(rng.uniform(0, mant + 8))) for _ in range(2)), reverse=True)
        taus = [2.0 ** top] + [t for t in taus if t < 2.0 ** top]
        if len(set(taus)) != len(taus):
            continue
        got, _, _ = oracle_strings(x, taus)
        modes, _ = model_brick(x, taus, dt)
        assert [m[2] for m in modes] == got
        modes_seen |= {m[0] for m in modes}
    assert MODE_CODED in modes_seen
