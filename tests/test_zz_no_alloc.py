"""pc_compress_noalloc, the allocation-free variant of pc_compress for callers
that cannot allocate device memory while they run: called through the C ABI
twice in a row on different fields, its streams must equal pc_compress's bit
for bit (the tolerance every stream comparison in these tests uses), and an
input beyond its fixed scratch must be refused before any GPU work."""
import ctypes as C

import numpy as np
import pytest

import synth_fields as S
from tests.gpu_helpers import parse_serialized

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    import paper_2308_11759_gb300 as pcz

    L = pcz.lib()
    fn = L.pc_compress_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.c_int, C.c_int, C.POINTER(C.c_double), C.c_int,
                   C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.POINTER(C.c_uint64),
                   C.POINTER(C.c_uint64), C.c_void_p]
    return pcz


def _noalloc(pcz, xd, tau, cap_words):
    shape = tuple(xd.shape)
    dims = (C.c_int64 * 3)(*shape[::-1])
    nb = [(d + 3) // 4 for d in shape[::-1]]
    nbricks = nb[0] * nb[1] * nb[2]
    nchunks = (nbricks + 31) // 32
    n = len(tau)
    # the caller owns the outputs; the entry point itself allocates nothing
    payload = torch.zeros(cap_words, dtype=torch.int64, device="cuda")
    chunk_word = torch.zeros(n * nchunks, dtype=torch.int64, device="cuda")
    brick_len = torch.zeros(n * nbricks, dtype=torch.int16, device="cuda")
    words = (C.c_uint64 * n)()
    counts = (C.c_uint64 * (5 * n))()
    taus = (C.c_double * n)(*tau)
    dt = pcz.PC_F32 if xd.dtype == torch.float32 else pcz.PC_F64
    rc = pcz.lib().pc_compress_noalloc(xd.data_ptr(), dims, 3, dt, taus, n, payload.data_ptr(), cap_words,
                                       chunk_word.data_ptr(), brick_len.data_ptr(), words, counts,
                                       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return rc, payload, chunk_word, brick_len, [int(w) for w in words], [int(c) for c in counts], nchunks, nbricks


def _check_same_as_pc_compress(pcz, x, tau):
    xd = torch.from_numpy(x).cuda()
    ref = parse_serialized(pcz.compress(xd, tau).serialize())
    need = sum(c["words"] for c in ref["comps"])
    rc, payload, cw, bl, words, counts, nch, nbr = _noalloc(pcz, xd, tau, need + 7)
    assert rc == 0, pcz.lib().pc_last_error()
    pay = payload.cpu().numpy().view(np.uint64)
    cwn = cw.cpu().numpy().view(np.uint64)
    bln = bl.cpu().numpy().view(np.uint16)
    base = 0
    for i, c in enumerate(ref["comps"]):
        assert words[i] == c["words"]
        assert np.array_equal(pay[base:base + words[i]], c["payload"]), f"payload of component {i + 1}"
        assert np.array_equal(cwn[i * nch:(i + 1) * nch], c["chunk_word"])
        assert np.array_equal(bln[i * nbr:(i + 1) * nbr], c["brick_len"])
        assert counts[5 * i:5 * i + 5] == c["counts"]
        base += words[i]


def _tau(x, kind, n):
    r = float(np.float64(x.max()) - np.float64(x.min()))
    if kind == "bin4":
        return [r * 2.0 ** (-4 * i) for i in range(1, n + 1)]
    return [float("1e-%d" % (i + 1)) * r for i in range(1, n + 1)]


def test_noalloc_equals_pc_compress_on_consecutive_calls(P):
    a = S.gaussians((64, 64, 64), seed=1)
    b = S.powerlaw((45, 38, 33), seed=2, dtype=np.float32)
    # two calls in a row on different fields and types (the shared scratch keeps
    # the previous call's contents), then the first field again
    _check_same_as_pc_compress(P, a, _tau(a, "bin4", 4))
    _check_same_as_pc_compress(P, b, _tau(b, "dec", 8))
    _check_same_as_pc_compress(P, a, _tau(a, "bin4", 4))


def test_noalloc_allocates_no_device_memory(P):
    # after a first call (which looks up the library array's address), a second
    # call of the same size leaves the device's free memory exactly as it was
    x = S.gaussians((48, 40, 36), seed=4)
    xd = torch.from_numpy(x).cuda()
    tau = _tau(x, "bin4", 4)
    shape = tuple(xd.shape)
    nb = [(d + 3) // 4 for d in shape[::-1]]
    nbricks = nb[0] * nb[1] * nb[2]
    nchunks = (nbricks + 31) // 32
    cap = 4 * nbricks * 140 + 64
    payload = torch.zeros(cap, dtype=torch.int64, device="cuda")
    chunk_word = torch.zeros(4 * nchunks, dtype=torch.int64, device="cuda")
    brick_len = torch.zeros(4 * nbricks, dtype=torch.int16, device="cuda")
    words = (C.c_uint64 * 4)()
    counts = (C.c_uint64 * 20)()
    taus = (C.c_double * 4)(*tau)
    dims = (C.c_int64 * 3)(*shape[::-1])

    def call():
        rc = P.lib().pc_compress_noalloc(xd.data_ptr(), dims, 3, P.PC_F64, taus, 4, payload.data_ptr(), cap,
                                         chunk_word.data_ptr(), brick_len.data_ptr(), words, counts,
                                         torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        return rc

    assert call() == 0
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    assert call() == 0
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_reserved() == reserved0


def test_noalloc_size_bound_is_exact(P):
    # the bound the refusal states is accepted, one chunk more is refused
    xd = torch.zeros(8, device="cuda", dtype=torch.float64)
    dims = (C.c_int64 * 3)(1024, 1024, 1024)
    words = (C.c_uint64 * 1)()
    counts = (C.c_uint64 * 5)()
    taus = (C.c_double * 1)(0.5)
    rc = P.lib().pc_compress_noalloc(xd.data_ptr(), dims, 3, P.PC_F64, taus, 1, xd.data_ptr(), 1, xd.data_ptr(),
                                     xd.data_ptr(), words, counts, None)
    msg = P.lib().pc_last_error().decode()
    assert rc == 1
    bound = int(msg.split("<=")[1].split()[0])  # chunks of one component
    assert 2000 <= bound <= 2100
    x = S.powerlaw((4, 4, 4 * 32 * bound), seed=6, dtype=np.float64)  # exactly `bound` chunks
    _check_same_as_pc_compress(P, x, [0.5])
    dims = (C.c_int64 * 3)(4 * 32 * (bound + 1), 4, 4)
    rc = P.lib().pc_compress_noalloc(xd.data_ptr(), dims, 3, P.PC_F64, taus, 1, xd.data_ptr(), 1, xd.data_ptr(),
                                     xd.data_ptr(), words, counts, None)
    assert rc == 1 and "scratch" in P.lib().pc_last_error().decode()


def test_noalloc_refuses_host_pointers(P):
    x = np.zeros((8, 8, 8))
    dims = (C.c_int64 * 3)(8, 8, 8)
    words = (C.c_uint64 * 1)()
    counts = (C.c_uint64 * 5)()
    taus = (C.c_double * 1)(0.5)
    d = torch.zeros(1024, device="cuda", dtype=torch.int64)
    rc = P.lib().pc_compress_noalloc(x.ctypes.data, dims, 3, P.PC_F64, taus, 1, d.data_ptr(), 1024, d.data_ptr(),
                                     d.data_ptr(), words, counts, None)
    assert rc == 1 and b"device memory" in P.lib().pc_last_error()


def test_noalloc_refuses_inputs_beyond_its_scratch(P):
    xd = torch.zeros(8, device="cuda", dtype=torch.float64)
    dims = (C.c_int64 * 3)(256, 256, 256)  # 262144 bricks: beyond the fixed scratch
    words = (C.c_uint64 * 4)()
    counts = (C.c_uint64 * 20)()
    taus = (C.c_double * 4)(1.0, 0.5, 0.25, 0.125)
    rc = P.lib().pc_compress_noalloc(xd.data_ptr(), dims, 3, P.PC_F64, taus, 4, xd.data_ptr(), 1, xd.data_ptr(),
                                     xd.data_ptr(), words, counts, None)
    assert rc == 1  # PC_ERR_ARG
    assert b"scratch" in P.lib().pc_last_error()
    # a payload buffer that is too small is refused with the size needed
    x = S.gaussians((16, 16, 16), seed=3)
    rc, *_ = _noalloc(P, torch.from_numpy(x).cuda(), _tau(x, "bin4", 3), 1)
    assert rc == 1 and b"need" in P.lib().pc_last_error()
