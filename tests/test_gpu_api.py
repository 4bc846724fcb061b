"""The C ABI on the GPU beyond the coder's bits: computed tolerances (Sec. 4.3)
equal the oracle's, the query on them, serialization round trips and the
checks on corrupt data, host-buffer calls, and every error status."""
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
    ("pl3d_f32", lambda: S.powerlaw((40, 36, 33), seed=31, dtype=np.float32), 8),
    ("fronts3d_f64", lambda: S.fronts((24, 20, 28), seed=32), 12),
    ("pl2d_f64", lambda: S.powerlaw((70, 51), seed=33, dtype=np.float64), 8),
    ("pl1d_f32", lambda: S.powerlaw((999,), seed=34, dtype=np.float32), 6),
    ("lossless3d_f64", lambda: _in_6_14(S.powerlaw((12, 10, 9), seed=21, dtype=np.float64)), 16),
]


def _in_6_14(f):
    """values in [6, 14]: the binary schedule's last tolerances lie below every ulp."""
    return 10.0 + 4.0 * f / np.abs(f).max()


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def pair(request, P):
    _, make, n = request.param
    x = np.ascontiguousarray(make())
    tau = O.tau_binary(O.value_range(x), 4, n) if "lossless" in request.param[0] else \
        O.tau_decade(O.value_range(x), n, first_exp=1)
    st = P.compress(torch.from_numpy(x).cuda(), tau)
    return x, tau, st, O.Streams(x, tau, nthreads=4)


def test_measured_errors_equal_oracle(pair):
    x, tau, st, ref = pair
    for i in range(st.n):
        m = st.measured_error(i)
        assert m == ref.measured(i), i
        assert m <= tau[i]
        got = st.retrieve(k=i + 1).cpu().numpy()
        assert m == float(np.max(np.abs(np.subtract(x, got, dtype=x.dtype))))


def test_query_on_measured_errors(pair):
    x, tau, st, ref = pair
    meas = [st.measured_error(i) for i in range(st.n)]
    rng = np.random.default_rng(8)
    for t in tau[0] * 10.0 ** (-rng.uniform(0.0, 14.0, 30)):
        if t < min(meas):
            with pytest.raises(Exception):
                st.query_k(t, measured=True)
            continue
        k = st.query_k(t, measured=True)
        assert k == O.query_k(meas, t)
        if t >= tau[-1]:
            assert k <= st.query_k(t)


def test_lossless_where_measured_error_is_zero(P):
    x = _in_6_14(S.powerlaw((12, 10, 9), seed=21, dtype=np.float64))
    tau = O.tau_binary(O.value_range(x), 4, 16)
    st = P.compress(torch.from_numpy(x).cuda(), tau)
    meas = [st.measured_error(i) for i in range(st.n)]
    k0 = next(i + 1 for i, m in enumerate(meas) if m == 0.0)
    assert torch.equal(st.retrieve(k=k0).cpu().view(torch.uint8), torch.from_numpy(x).view(torch.uint8))
    assert st.query_k(0.0, measured=True) == k0


def test_serialize_round_trip(P, pair):
    x, tau, st, ref = pair
    blob = st.serialize()
    d = parse_serialized(blob)
    assert d["version"] == 2
    for i in range(st.n):
        assert d["comps"][i]["measured"] == st.measured_error(i)
    st2 = P.Streams.deserialize(blob)
    assert st2.shape == st.shape and st2.n == st.n
    assert st2.serialize() == blob
    for k in (1, st.n):
        assert torch.equal(st2.retrieve(k=k).view(torch.uint8), st.retrieve(k=k).view(torch.uint8))
    for i in range(st.n):
        assert st2.measured_error(i) == st.measured_error(i)
        assert st2.counts(i) == st.counts(i)


def _status(fn):
    with pytest.raises(Exception) as e:
        fn()
    return getattr(e.value, "name", None)


def test_corrupt_streams_are_rejected(P, pair):
    x, tau, st, ref = pair
    blob = bytearray(st.serialize())
    bad = bytearray(blob)
    bad[4] = 1  # format version 1
    assert _status(lambda: P.Streams.deserialize(bytes(bad))) == "PC_ERR_VERSION"
    bad = bytearray(blob)
    bad[0] ^= 0xFF  # magic
    assert _status(lambda: P.Streams.deserialize(bytes(bad))) == "PC_ERR_VERSION"
    assert _status(lambda: P.Streams.deserialize(bytes(blob[:-8]))) == "PC_ERR_CORRUPT_STREAM"
    d = parse_serialized(bytes(blob))
    n, nch, nbr = d["n"], d["nchunks"], d["nbricks"]
    # the first brick length of component 1 made one bit longer: its block no longer parses
    bl_off = 64 + 64 * n + 8 * nch
    bad = bytearray(blob)
    v = int.from_bytes(bad[bl_off:bl_off + 2], "little")
    bad[bl_off:bl_off + 2] = (v + 1).to_bytes(2, "little")
    assert _status(lambda: P.Streams.deserialize(bytes(bad))) == "PC_ERR_CORRUPT_STREAM"
    bad = bytearray(blob)
    bad[64 + 56:64 + 64] = np.float64(-1.0).tobytes()  # a negative measured error
    assert _status(lambda: P.Streams.deserialize(bytes(bad))) == "PC_ERR_CORRUPT_STREAM"
    bad = bytearray(blob)
    bad[64:72] = np.float64(tau[1]).tobytes() if n > 1 else np.float64(-1.0).tobytes()  # tau no longer decreasing
    assert _status(lambda: P.Streams.deserialize(bytes(bad))) == "PC_ERR_CORRUPT_STREAM"


def test_host_buffers(P):
    x = S.powerlaw((21, 19, 17), seed=35, dtype=np.float32)
    tau = O.tau_decade(O.value_range(x), 5)
    dev = P.compress(torch.from_numpy(x).cuda(), tau)
    host = P.compress(x, tau)  # the library copies the field in
    assert host.serialize() == dev.serialize()
    out = np.empty_like(x)
    host.retrieve(k=3, out=out)
    assert np.array_equal(out.view(np.uint8), dev.retrieve(k=3).cpu().numpy().view(np.uint8))
    part = np.empty((5, 6, 7), dtype=np.float32)
    host.retrieve(k=4, box=([3, 2, 1], [8, 8, 8]), out=part)
    assert np.array_equal(part, dev.retrieve(k=4).cpu().numpy()[3:8, 2:8, 1:8])
    # pinned host memory: read and written in place by the kernels
    xp = torch.from_numpy(x).pin_memory()
    pinned = P.compress(xp, tau)
    assert pinned.serialize() == dev.serialize()
    assert P.field_range(xp) == P.field_range(torch.from_numpy(x).cuda())
    op = torch.empty(x.shape, dtype=torch.float32).pin_memory()
    pinned.retrieve(k=3, out=op)
    torch.cuda.synchronize()  # pinned results are complete in stream order
    assert torch.equal(op.view(torch.uint8), dev.retrieve(k=3).cpu().view(torch.uint8))
    acc = torch.empty(x.shape, dtype=torch.float32).pin_memory()
    pinned.retrieve(k=2, out=acc)
    pinned.refine(2, 5, acc)  # x~_2 read from and x~_5 written to pinned memory
    torch.cuda.synchronize()
    assert torch.equal(acc.view(torch.uint8), dev.retrieve(k=5).cpu().view(torch.uint8))
    # 2D and 1D fields: pinned input and output (written in place by the kernel), pageable output
    for shape, dt in (((130, 97), np.float64), ((4099,), np.float32)):
        y = S.powerlaw(shape, seed=36, dtype=dt)
        t = O.tau_decade(O.value_range(y), 6)
        d = P.compress(torch.from_numpy(y).cuda(), t)
        h = P.compress(torch.from_numpy(y).pin_memory(), t)
        assert h.serialize() == d.serialize()
        want = d.retrieve(k=4).cpu()
        o1 = torch.empty(want.shape, dtype=want.dtype).pin_memory()
        h.retrieve(k=4, out=o1)
        o2 = np.empty(shape, dtype=dt)
        h.retrieve(k=4, out=o2)  # pageable: returns with the data in place
        torch.cuda.synchronize()
        assert torch.equal(o1.view(torch.uint8), want.view(torch.uint8))
        assert np.array_equal(o2.view(np.uint8), want.numpy().view(np.uint8))


def test_error_statuses(P):
    x = S.powerlaw((9, 8, 7), seed=36, dtype=np.float64)
    xd = torch.from_numpy(x).cuda()
    tau = [0.1, 0.01, 0.001]
    for bad_val in (np.nan, np.inf, -np.inf):
        y = x.copy()
        y[4, 3, 2] = bad_val
        assert _status(lambda: P.compress(torch.from_numpy(y).cuda(), tau)) == "PC_ERR_NONFINITE"
    assert _status(lambda: P.compress(xd, [0.1, 0.2])) == "PC_ERR_TAU_ORDER"
    assert _status(lambda: P.compress(xd, [0.1, 0.0])) == "PC_ERR_TAU_ORDER"
    assert _status(lambda: P.compress(xd, [0.1, float("nan")])) == "PC_ERR_TAU_ORDER"
    assert _status(lambda: P.compress(xd, [])) == "PC_ERR_ARG"
    st = P.compress(xd, tau)
    assert _status(lambda: st.query_k(1e-4)) == "PC_ERR_TOL_UNREACHABLE"
    assert _status(lambda: st.retrieve(tau=1e-4)) == "PC_ERR_TOL_UNREACHABLE"
    assert _status(lambda: st.retrieve(k=4)) == "PC_ERR_ARG"
    assert _status(lambda: st.retrieve(k=1, box=([0, 0, 0], [10, 8, 7]))) == "PC_ERR_ARG"
    assert _status(lambda: st.retrieve(k=1, box=([3, 0, 0], [3, 8, 7]))) == "PC_ERR_ARG"
    assert _status(lambda: st.refine(2, 1, torch.empty_like(xd))) == "PC_ERR_ARG"
    assert st.query_k(0.5) == 1 and st.query_k(0.01) == 2
    z = st.retrieve(k=0).cpu().numpy()
    assert not z.any()


def test_lossless_sweep(P):
    """Sec. 5.1.3 on a float32 and a float64 field: the sweep's k reproduces x
    bit for bit, k - 1 does not, and the rate is the streams' own."""
    for dt, shape in ((np.float32, (20, 18, 16)), (np.float64, (48, 40))):
        x = S.powerlaw(shape, seed=37, dtype=dt)
        xd = torch.from_numpy(x).cuda()
        r = P.lossless_sweep(xd, delta=4)
        k, st = r["k"], r["streams"]
        assert k is not None
        assert torch.equal(st.retrieve(k=k).view(torch.uint8), xd.view(torch.uint8))
        assert not torch.equal(st.retrieve(k=k - 1), xd)
        bits = sum(st.info(i)[1] + 8 * st.info(i)[2] for i in range(k)) / x.size
        assert r["bits_per_value"] == bits and r["ratio"] == 8 * x.itemsize / bits
        ref = O.Streams(x, [st.tau(i) for i in range(st.n)], nthreads=4)
        assert [ref.measured(i) for i in range(st.n)] == r["measured"]


def test_pinned_output_by_slabs(P):
    """A retrieval of 32 MiB or more into pinned host memory goes through device
    staging slabs of whole brick layers (about 64 MiB each) and the copy
    engines: a 320x256x258 float64 field (169 MB, three slabs, so each staging
    buffer is reused).  The result, read after the stream is synchronised,
    equals the device retrieval for the full box, for a sub-box whose first
    slab starts inside a brick layer, and for a refinement read from and
    written to pinned memory."""
    x = S.powerlaw((320, 256, 258), seed=44, dtype=np.float64)
    tau = O.tau_decade(O.value_range(x), 6)
    st = P.compress(torch.from_numpy(x).cuda(), tau)
    for k in (1, 6):
        out = torch.empty(x.shape, dtype=torch.float64).pin_memory()
        st.retrieve(k=k, out=out)
        torch.cuda.synchronize()
        assert torch.equal(out.view(torch.uint8), st.retrieve(k=k).cpu().view(torch.uint8))
    box = ([3, 1, 2], [317, 256, 257])
    part = torch.empty((314, 255, 255), dtype=torch.float64).pin_memory()
    st.retrieve(k=4, box=box, out=part)
    torch.cuda.synchronize()
    assert torch.equal(part.view(torch.uint8), st.retrieve(k=4, box=box).cpu().view(torch.uint8))
    acc = torch.empty(x.shape, dtype=torch.float64).pin_memory()
    st.retrieve(k=2, out=acc)
    st.refine(2, 5, acc)
    torch.cuda.synchronize()
    assert torch.equal(acc.view(torch.uint8), st.retrieve(k=5).cpu().view(torch.uint8))


def test_release_cached_memory(P):
    """Freed streams and scratch stay in the library's pools for later calls;
    pc_release_cached_memory hands them back to the driver, leaves live
    streams usable, and later calls rebuild the pools on demand."""
    x = S.powerlaw((96, 96, 96), seed=45, dtype=np.float64)
    xd = torch.from_numpy(x).cuda()
    tau = O.tau_decade(O.value_range(x), 5)
    live = P.compress(xd, tau)
    gone = P.compress(xd, tau)
    ref = gone.retrieve(k=3).cpu()
    gone.close()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    P.release_cached_memory()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 > free0  # at least the construction bit pool went back
    assert torch.equal(live.retrieve(k=3).cpu(), ref)
    again = P.compress(xd, tau)
    assert torch.equal(again.retrieve(k=3).cpu(), ref)
    again.close()
    live.close()


def test_free_waits_for_its_own_work_only(P):
    """pc_streams_free waits for the library's launches that read the streams,
    on whatever stream they were queued, and not for unrelated work: (1) a
    retrieval queued behind a backlog on one stream, then the streams freed
    at once and their memory reused by another field's streams, still reads
    intact streams; (2) freeing streams returns while another stream's
    backlog is still running."""
    x = S.powerlaw((192, 192, 192), seed=46, dtype=np.float32)
    xd = torch.from_numpy(x).cuda()
    tau = O.tau_decade(O.value_range(x), 8)
    ref = P.compress(xd, tau)
    want = ref.retrieve(k=8)
    torch.cuda.synchronize()
    a = torch.randn(8192, 8192, device="cuda")
    sB, sC, sD = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    st = P.compress(xd, tau)
    out = torch.empty_like(xd)
    with torch.cuda.stream(sB):
        b = a
        for _ in range(8):
            b = b @ a
        st.retrieve(k=8, out=out, stream=sB)
    st.close()  # returns once the retrieval on sB has run
    y = torch.from_numpy(S.gaussians((192, 192, 192), seed=47, dtype=np.float32)).cuda()
    torch.cuda.synchronize()
    other = P.compress(y, tau, stream=sD)  # takes the freed pool blocks
    sD.synchronize()
    assert torch.equal(out.view(torch.int32), want.view(torch.int32))
    with torch.cuda.stream(sC):
        c = a
        for _ in range(20):
            c = c @ a
    other.close()
    assert not sC.query()  # the backlog on sC did not hold the free up
    torch.cuda.synchronize()
    ref.close()


def test_calls_from_fresh_threads_on_their_own_streams(P):
    """Each host thread (whose first CUDA call is the library's) runs one
    field's pipeline -- range and schedule, compress and retrievals -- on its
    own stream, from pinned host memory into pinned host memory; the results
    equal the same calls made one after the other on the default stream."""
    import threading

    # the first output (42 MB) goes through the staging slabs, the second (7 MB) is written in place
    xs = [S.powerlaw((256, 256, 160), seed=48, dtype=np.float32), S.fronts((96, 100, 90), seed=49)]
    hin = [torch.from_numpy(x).pin_memory() for x in xs]
    want = []
    for h in hin:
        st = P.compress(h, P.field_tau_schedule(h, "decade", 6))
        want.append([st.retrieve(k=k).cpu() for k in (2, 6)])
        st.close()
    got = [None, None]
    errors = []

    def run(j):
        try:
            s = torch.cuda.Stream()
            tau = P.field_tau_schedule(hin[j], "decade", 6, stream=s)
            st = P.compress(hin[j], tau, stream=s)
            outs = [torch.empty(hin[j].shape, dtype=hin[j].dtype).pin_memory() for _ in range(2)]
            for o, k in zip(outs, (2, 6)):
                st.retrieve(k=k, out=o, stream=s)
            s.synchronize()
            st.close()
            got[j] = outs
        except Exception as e:  # reported below
            errors.append(e)

    threads = [threading.Thread(target=run, args=(j,)) for j in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for j in range(2):
        for o, w in zip(got[j], want[j]):
            assert torch.equal(o.view(torch.uint8), w.view(torch.uint8))
