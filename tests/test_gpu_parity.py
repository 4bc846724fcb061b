"""GPU path vs the CPU oracle, through the C ABI: the component streams (payload,
index, block counters) and every reconstruction must be bit-identical, at
sizes that span many chunks and ragged edges."""
import numpy as np
import pytest

import oracle as O
import synth_fields as S
from tests.gpu_helpers import parse_serialized

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    import paper_2308_11759_gb300 as pcz

    pcz.lib()
    return pcz


CASES = [
    ("gauss64_f64_delta4", lambda: S.gaussians((64, 64, 64), seed=1), "bin4", 4),
    ("gauss64_f32_delta4", lambda: S.gaussians((64, 64, 64), seed=1, dtype=np.float32), "bin4", 4),
    ("pl_f32_ragged_decade", lambda: S.powerlaw((45, 38, 33), seed=2, dtype=np.float32), "dec", 8),
    ("pl_f64_ragged_decade", lambda: S.powerlaw((45, 38, 33), seed=2, dtype=np.float64), "dec", 8),
    ("fronts_f64_12", lambda: S.fronts((28, 24, 21), seed=5), "dec", 12),
    ("fronts_f32_12", lambda: S.fronts((28, 24, 21), seed=5, dtype=np.float32), "dec", 12),
    ("lossless_f64_14", lambda: (10.0 + 4.0 * S.powerlaw((12, 10, 9), seed=21, dtype=np.float64)), "bin4", 14),
    ("tiny_1x1x1", lambda: np.array([[[3.25]]]), None, 3),
    ("thin_3x5x130_f32", lambda: S.powerlaw((3, 5, 130), seed=9, dtype=np.float32), "bin4", 5),
    ("constant", lambda: np.full((9, 8, 7), 1.5), None, 3),
    ("zeros", lambda: np.zeros((8, 8, 8), dtype=np.float32), None, 2),
    # white noise: every coefficient significant within the top planes, so a
    # plane's group-test part runs past one 64-bit window and the last
    # coefficient turns significant inside a decoded byte
    ("noise_f32_dense", lambda: _noise((22, 21, 20), 31, np.float32, 0), "dec", 6),
    # magnitudes spread over 2^-40..1 within each brick, with exact zeros
    ("noise_f64_wide", lambda: _noise((19, 18, 17), 32, np.float64, 40), "bin8", 8),
    # 2D and 1D fields (4x4 and 4-value bricks)
    ("pl2d_f32_ragged_decade", lambda: S.powerlaw((157, 389), seed=12, dtype=np.float32), "dec", 8),
    ("pl2d_f64_bin4", lambda: S.powerlaw((130, 97), seed=13, dtype=np.float64), "bin4", 10),
    ("gauss2d_f64_decade", lambda: S.gaussians((64, 64), seed=14), "dec", 8),
    ("steps2d_f32_12", lambda: _steps((75, 66), 15, np.float32), "dec", 12),
    ("steps2d_f64_12", lambda: _steps((75, 66), 15, np.float64), "dec", 12),
    ("lossless2d_f32_14", lambda: (10.0 + 4.0 * S.powerlaw((23, 21), seed=22, dtype=np.float32)), "bin4", 14),
    ("pl1d_f64_decade", lambda: S.powerlaw((4099,), seed=16, dtype=np.float64), "dec", 8),
    ("pl1d_f32_bin4", lambda: S.powerlaw((1001,), seed=17, dtype=np.float32), "bin4", 6),
    ("tiny1d_3", lambda: np.array([1.0, 2.0, 7.0]), None, 3),
    ("thin2d_1x70_f32", lambda: S.powerlaw((1, 70), seed=18, dtype=np.float32), "bin4", 5),
    # Eq. 1 enforcement (Sec. 4.3): every brick RAW (float32 noise, one component
    # below what its block exponent can code)
    ("raw_noise_f32_one", lambda: np.random.default_rng(31).uniform(-1, 1, size=(24, 20, 18)).astype(np.float32),
     [2.0 ** -26], 1),
    # RAW and CODED bricks side by side in one warp, and the violations that
    # floating point leaves where x~_1 is far from small values of x
    ("viol_f32_3d", lambda: _wide((21, 19, 18), 33, np.float32), [0.25, 2.0 ** -30], 2),
    ("viol_f64_3d", lambda: _wide((21, 19, 18), 34, np.float64), [0.25, 2.0 ** -59], 2),
    ("viol_f32_1d", lambda: _wide((2051,), 35, np.float32), [0.25, 2.0 ** -30], 2),
    ("viol_f64_2d", lambda: _wide((37, 41), 36, np.float64), [0.25, 2.0 ** -59], 2),
    # the top of the float range: reconstructions round to infinity, the coder
    # escalates and stores some bricks RAW
    ("top_f32_bin", lambda: _top(np.float32, 0.9999, (18, 17, 16)), "bin4", 6),
    ("top_f32_dec", lambda: _top(np.float32, 0.999, (18, 17, 16)), "dec", 6),
    ("top_f64_bin", lambda: _top(np.float64, 0.9, (18, 17, 16)), "bin4", 6),
    ("top2d_f64_dec", lambda: _top(np.float64, 0.99, (45, 38)), "dec", 6),
    ("top1d_f32_bin", lambda: _top(np.float32, 0.9999, (1003,)), "bin4", 6),
    # scales where quantisation and dequantisation leave the normal-range fast
    # paths: subnormal values, residuals near 2^-100 (float32) and near the top
    ("scaled_f32_1e-40", lambda: _scaled(1e-40, np.float32), "dec", 8),
    ("scaled_f32_1e-36", lambda: _scaled(1e-36, np.float32), "dec", 8),
    ("scaled_f32_1e37", lambda: _scaled(1e37, np.float32), "dec", 8),
    ("scaled_f64_1e-310", lambda: _scaled(1e-310, np.float64), "dec", 8),
    ("scaled_f64_1e306", lambda: _scaled(1e306, np.float64), "dec", 8),
    # 1D bricks that escalate (every third brick; stored inputs), mixed with random bricks
    ("esc1d_f32", lambda: _esc1d(0, 257, 50)[0], lambda: _esc1d(0, 257, 50)[1], 2),
    ("esc1d_f64", lambda: _esc1d(3, 257, 51)[0], lambda: _esc1d(3, 257, 51)[1], 2),
    # the largest component count (PC_MAX_COMPONENTS = 64, tau_i = 2^-i range): retrieval in
    # 8 rounds of 8 components, the late components lossless or ZERO
    ("max64_f64_bin1", lambda: S.powerlaw((14, 13, 11), seed=23, dtype=np.float64), "bin1", 64),
    ("max64_f32_bin1", lambda: S.powerlaw((14, 13, 11), seed=24, dtype=np.float32), "bin1", 64),
    ("max64_2d_f32_bin1", lambda: S.powerlaw((37, 29), seed=25, dtype=np.float32), "bin1", 64),
]


def _wide(shape, seed, dtype):
    """N(0, 1) values each scaled by 2^-U(0, 8)."""
    rng = np.random.default_rng(seed)
    return (rng.normal(size=shape) * 2.0 ** rng.uniform(-8, 0, size=shape)).astype(dtype)


def _top(dtype, frac, shape, seed=7):
    """magnitudes in [frac, 1] of the largest finite value, signs of a k^-5/3 field
    (one-signed for float64, so that the range max - min stays finite)."""
    base = S.powerlaw(shape, seed=seed, dtype=np.float64)
    base = base / np.abs(base).max()
    mag = (frac + (1 - frac) * np.abs(base)) * float(np.finfo(dtype).max)
    return (mag if dtype == np.float64 else np.sign(base) * mag).astype(dtype)


def _scaled(scale, dtype):
    return (S.powerlaw((20, 18, 17), seed=4, dtype=np.float64) * scale).astype(dtype)


def _esc1d(row, nbricks, seed):
    """every third brick the stored escalating brick of tests/golden/escalation_1d.txt
    (row `row`), the others random; a ragged tail of 3 values.  Returns (x, tau)."""
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "escalation_1d.txt")
    rows = [[p.strip() for p in ln.split("|")] for ln in open(path) if ln.strip() and not ln.startswith("#")]
    dtn, hexes, taus = rows[row]
    dtype = np.float32 if dtn == "f32" else np.float64
    ints = np.array([int(h, 16) for h in hexes.split(",")], dtype=np.uint32 if dtype == np.float32 else np.uint64)
    brick = ints.view(dtype)
    rng = np.random.default_rng(seed)
    parts = [brick if j % 3 == 0 else (rng.normal(size=4) * 2.0 ** rng.uniform(-3, 3, size=4)).astype(dtype)
             for j in range(nbricks)]
    return np.concatenate(parts + [brick[:3]]), [float.fromhex(t) for t in taus.split()]


def _steps(shape, seed, dtype):
    """powerlaw plus jumps of height 3 where it crosses 0.5 (sharp fronts)."""
    f = S.powerlaw(shape, seed=seed, dtype=np.float64)
    return (f + np.where(f > 0.5, 3.0, 0.0)).astype(dtype)


def _noise(shape, seed, dtype, spread):
    """uniform noise in (-1, 1), each value scaled by 2^-U{0..spread}; one value in 16 is 0."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(-1.0, 1.0, size=shape) * np.exp2(-rng.integers(0, spread + 1, size=shape))
    f[rng.random(shape) < 1.0 / 16] = 0.0
    return f.astype(dtype)


def _tau(x, kind, n):
    if callable(kind):
        return kind()
    if isinstance(kind, list):
        return kind
    if kind is None:
        return [1.0 / (i + 1) for i in range(n)]
    r = O.value_range(x)
    if kind in ("bin1", "bin8"):
        return O.tau_binary(r, int(kind[3:]), n)
    return O.tau_binary(r, 4, n) if kind == "bin4" else O.tau_decade(r, n)


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def pair(request, P):
    _, make, kind, n = request.param
    x = np.ascontiguousarray(make())
    tau = _tau(x, kind, n)
    xd = torch.from_numpy(x).cuda()
    if isinstance(kind, str):  # the product's own schedule from the device range is the oracle's, bit for bit
        if kind.startswith("bin"):
            gt = P.field_tau_schedule(xd, "binary", n, param=int(kind[3:]))
        else:
            gt = P.field_tau_schedule(xd, "decade", n)
        assert gt == tau
    gpu = P.compress(xd, tau)
    ref = O.Streams(x, tau, nthreads=4)
    return x, tau, gpu, ref


def test_streams_bitwise(pair):
    x, tau, gpu, ref = pair
    d = parse_serialized(gpu.serialize())
    assert d["n"] == ref.n and d["nbricks"] == ref.nbricks and d["nchunks"] == ref.nchunks
    for i in range(ref.n):
        c = d["comps"][i]
        assert c["tau"] == tau[i]
        assert np.array_equal(c["brick_len"], ref.brick_len(i)), f"brick lengths of component {i + 1}"
        assert np.array_equal(c["chunk_word"], ref.chunk_word(i)), f"chunk offsets of component {i + 1}"
        assert np.array_equal(c["payload"], ref.payload(i)), f"payload of component {i + 1}"
        assert c["counts"] == [int(v) for v in ref.stats(i)]
        assert gpu.counts(i) == c["counts"]


def test_retrieve_bitwise_and_eq1(pair):
    x, tau, gpu, ref = pair
    for k in range(0, ref.n + 1):
        got = gpu.retrieve(k=k).cpu().numpy()
        want = ref.retrieve(k)
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), f"k={k}"
        if k:  # Eq. 1, with the violations floating point leaves counted, not hidden
            err = np.abs(np.subtract(x, got, dtype=x.dtype)).astype(np.float64)
            assert int(np.sum(err > tau[k - 1])) == int(ref.stats(k - 1)[O.ST_VIOL])


def test_refine_equals_one_shot(pair):
    x, tau, gpu, ref = pair
    for k0 in range(0, ref.n):
        acc = gpu.retrieve(k=k0)
        for k in range(k0 + 1, ref.n + 1):
            gpu.refine(k - 1, k, acc)
            assert torch.equal(acc.view(torch.uint8), gpu.retrieve(k=k).view(torch.uint8))


def test_subbox(pair):
    x, tau, gpu, ref = pair
    rng = np.random.default_rng(3)
    k = (ref.n + 1) // 2
    full = gpu.retrieve(k=k).cpu().numpy()
    for _ in range(6):
        lo = [int(rng.integers(0, s)) for s in x.shape]
        hi = [int(rng.integers(l + 1, s + 1)) for l, s in zip(lo, x.shape)]
        part = gpu.retrieve(k=k, box=(lo, hi)).cpu().numpy()
        sl = tuple(slice(l, h) for l, h in zip(lo, hi))
        assert np.array_equal(part, full[sl])
        assert np.array_equal(part, ref.retrieve(k, box=(lo, hi)))


def test_query_by_tolerance(pair):
    x, tau, gpu, ref = pair
    for i, t in enumerate(tau):
        assert gpu.query_k(t) == i + 1
        got = gpu.retrieve(tau=t * 1.5).cpu().numpy()
        assert np.array_equal(got, ref.retrieve(O.query_k(tau, t * 1.5)))
