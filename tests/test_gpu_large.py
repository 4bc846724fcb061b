"""Parity at the full sizes of the benchmark workloads, in the launch
configuration bench.py times:

* 512^3 k^-5/3 field, float32 and float64, 8 components (decade schedule):
  every component's index and payload equal the oracle's bit for bit (the
  oracle codes the whole field on all host cores), block counters agree, Eq. 1
  holds at every k over the whole field, and sub-box retrievals equal the
  oracle's.
* 1024^3 float64 field with sharp fronts, 12 components down to 1e-12 * range:
  bricks sampled across the field (corners, edges, random) are coded by the
  oracle one at a time and compared bit for bit with the GPU streams, and the
  GPU reconstructions of those bricks at several k equal the oracle's; Eq. 1
  holds at every k over the whole field.
"""
import os

import numpy as np
import pytest

import oracle as O
import synth_fields as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    import paper_2308_11759_gb300 as pcz

    pcz.lib()
    return pcz


def _eq1_every_k(st, xd, tau):
    """max |fl_T(x - x~_k)| <= tau_k at every k, evaluated by torch in the field's precision."""
    out = torch.empty_like(xd)
    prev = float("inf")
    for k in range(1, st.n + 1):
        st.retrieve(k=k, out=out)
        err = (xd - out).abs().max().item()
        assert err <= tau[k - 1], (k, err, tau[k - 1])
        assert err <= prev
        prev = err


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_512_full_streams(P, dt):
    x64 = S.powerlaw((512, 512, 512), seed=2, dtype=np.float64, device="cuda")
    xd = (x64.float() if dt == "f32" else x64).contiguous()
    del x64
    x = xd.cpu().numpy()
    tau = O.tau_decade(O.value_range(x), 8)
    assert P.field_tau_schedule(xd, "decade", 8) == tau
    st = P.compress(xd, tau)
    ref = O.Streams(x, tau, nthreads=os.cpu_count() or 1)
    for i in range(8):
        cw, bl = st.read_index(i)
        assert np.array_equal(bl, ref.brick_len(i)), f"brick lengths of component {i + 1}"
        assert np.array_equal(cw, ref.chunk_word(i)), f"chunk offsets of component {i + 1}"
        nw = st.info(i)[1] // 64
        assert nw == len(ref.payload(i))
        assert np.array_equal(st.read_payload(i, 0, nw), ref.payload(i)), f"payload of component {i + 1}"
        assert st.counts(i) == [int(v) for v in ref.stats(i)]
        assert st.counts(i)[4] == 0
    _eq1_every_k(st, xd, tau)
    rng = np.random.default_rng(7)
    for k in (1, 4, 8):
        for _ in range(3):
            lo = [int(v) for v in rng.integers(0, 500, 3)]
            hi = [l + int(v) for l, v in zip(lo, rng.integers(1, 13, 3))]
            got = st.retrieve(k=k, box=(lo, hi)).cpu().numpy()
            want = ref.retrieve(k, box=(lo, hi))
            assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (k, lo, hi)


def test_1024_fronts_sampled(P):
    n = 12
    xd = S.fronts((1024, 1024, 1024), seed=5, dtype=np.float64, device="cuda")
    lo_v, hi_v = xd.min().item(), xd.max().item()
    rng_v = float(np.float64(hi_v) - np.float64(lo_v))
    tau = O.tau_decade(rng_v, n, first_exp=1)  # tau_i = 10^-i * range, i = 1..12
    assert P.field_tau_schedule(xd, "decade", n, param=1) == tau
    st = P.compress(xd, tau)
    for i in range(n):
        assert st.counts(i)[4] == 0
    nb = 256  # bricks per axis
    rs = np.random.default_rng(11)
    coords = [(0, 0, 0), (nb - 1, nb - 1, nb - 1), (nb - 1, 0, 0), (0, nb - 1, 0), (0, 0, nb - 1)]
    coords += [tuple(int(v) for v in rs.integers(0, nb, 3)) for _ in range(1500)]
    # the sampled bricks' values (4x4x4 each), gathered on the device
    idx = torch.tensor(coords, device="cuda", dtype=torch.int64)  # (bx, by, bz)
    ar = torch.arange(4, device="cuda")
    zz = (4 * idx[:, 2])[:, None, None, None] + ar[None, :, None, None]
    yy = (4 * idx[:, 1])[:, None, None, None] + ar[None, None, :, None]
    xx = (4 * idx[:, 0])[:, None, None, None] + ar[None, None, None, :]
    bricks = xd[zz, yy, xx].cpu().numpy()  # (S, 4, 4, 4) in (z, y, x) order
    index = [st.read_index(i) for i in range(n)]
    ref_bits = []
    for s_i, (bx, by, bz) in enumerate(coords):
        b = bx + nb * (by + nb * bz)
        bits, nbits, _, _ = O.code_brick(np.ascontiguousarray(bricks[s_i]), tau, 0, maxwords=160)
        ref_bits.append((bits, nbits))
        for i in range(n):
            v, L = st.brick_bits(i, b, index[i])
            assert L == int(nbits[i]), (b, i)
            assert v == O.bits_as_int(bits[i], nbits[i]), (b, i)
    out = torch.empty_like(xd)
    for k in (1, 5, 9, 12):
        st.retrieve(k=k, out=out)
        got = out[zz, yy, xx].cpu().numpy()
        for s_i in range(len(coords)):
            bits, nbits = ref_bits[s_i]
            want = O.decode_brick(np.float64, 3, tau, k, bits, nbits)
            assert np.array_equal(got[s_i].reshape(-1).view(np.uint64), want.view(np.uint64)), (coords[s_i], k)
    del out
    _eq1_every_k(st, xd, tau)
