"""The C ABI without a GPU: libpcz.so builds and loads, exports every function
include/pcz.h declares, the ctypes structures have the header's sizes, and
calls whose arguments are invalid fail with PC_ERR_ARG before any device work."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pcz.h")


@pytest.fixture(scope="module")
def L():
    from paper_2308_11759_gb300 import build as B

    try:
        B.build()
    except (RuntimeError, FileNotFoundError) as e:  # no CUDA toolkit on this machine
        pytest.skip(f"libpcz cannot be built here: {e}")
    import paper_2308_11759_gb300 as P

    return P.lib()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pc_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("pc_compress", "pc_retrieve", "pc_refine", "pc_query_k", "pc_query_k_measured",
                 "pc_stream_measured_error", "pc_streams_serialize", "pc_streams_deserialize", "pc_server_create",
                 "pc_server_replay", "pc_compress_noalloc", "pc_last_error", "pc_version"):
        assert want in names


def test_every_declared_function_is_exported(L):
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_struct_sizes(L):
    import paper_2308_11759_gb300 as P

    assert C.sizeof(P.Box) == 48
    assert C.sizeof(P.Query) == 64  # int, int, double, pc_box
    assert C.sizeof(P.ServeStats) == 64


def test_version_and_error_text(L):
    assert L.pc_version() == 2
    assert isinstance(L.pc_last_error(), bytes)


def test_argument_errors_without_device_work(L):
    import paper_2308_11759_gb300 as P

    k = C.c_int()
    assert L.pc_query_k(None, 1.0, C.byref(k)) == 1
    assert b"NULL" in L.pc_last_error()
    assert L.pc_query_k_measured(None, 1.0, C.byref(k)) == 1
    e = C.c_double()
    assert L.pc_stream_measured_error(None, 0, C.byref(e)) == 1
    h = C.c_void_p()
    dims = (C.c_int64 * 3)(4, 4, 4)
    tau = (C.c_double * 1)(1.0)
    assert L.pc_compress(None, dims, 3, 1, tau, 1, None, C.byref(h)) == 1
    assert L.pc_compress(None, dims, 3, 1, tau, 1, None, None) == 1
    srv = C.c_void_p()
    assert L.pc_server_create(1 << 30, 0, 0, None, C.byref(srv)) == 1  # max_batch < 1
    assert L.pc_server_create(1 << 30, 4, 8, None, C.byref(srv)) == 1  # unknown flag
    assert L.pc_server_free(None) == 0
    st = C.c_void_p()
    assert L.pc_streams_deserialize(None, 0, None, C.byref(st)) == 1
    buf = (C.c_ubyte * 16)()
    assert L.pc_streams_deserialize(buf, 16, None, C.byref(st)) == 8  # PC_ERR_VERSION: too short
    assert P.STATUS[8] == "PC_ERR_VERSION"


def test_tau_schedules_on_the_host(L):
    """pc_tau_schedule (pure host arithmetic, no GPU): each tolerance is the
    exact schedule value rounded once to double (Sec. 5.1), checked with exact
    rationals, and the values equal the oracle's own copy of the rule."""
    from fractions import Fraction

    import oracle as O
    import paper_2308_11759_gb300 as P

    for tau0 in (1.0, 3.7, 0.1234567, 2.5e-300, 1.7e308, 6.02e23):
        for delta in (1, 4, 8, 16):
            got = P.tau_binary(tau0, delta, 12)
            assert got == O.tau_binary(tau0, delta, 12)
            for i, t in enumerate(got, 1):
                assert t == float(Fraction(tau0) / 2 ** (delta * i))
        for first in (0, 1, 2, 7):
            got = P.tau_decade(tau0, 10, first_exp=first)
            assert got == O.tau_decade(tau0, 10, first_exp=first)
            for i, t in enumerate(got, 1):
                c = float(Fraction(1, 10 ** (first + i - 1)))  # the double nearest 10^-e
                assert t == float(Fraction(c) * Fraction(tau0))
    out = (C.c_double * 4)()
    assert L.pc_tau_schedule(P.PC_TAU_BINARY, -1.0, 4, 4, out) == 1
    assert L.pc_tau_schedule(P.PC_TAU_BINARY, float("inf"), 4, 4, out) == 1
    assert L.pc_tau_schedule(P.PC_TAU_BINARY, 1.0, 0, 4, out) == 1
    assert L.pc_tau_schedule(7, 1.0, 4, 4, out) == 1
    assert L.pc_tau_schedule(P.PC_TAU_DECADE, 1.0, 2, 0, out) == 1


def test_derivative_argument_errors_without_device_work(L):
    """pc_fd_vorticity_z / pc_fd_second refuse bad shapes, axes and spacings
    with PC_ERR_ARG before any device work (and host pointers after it)."""
    d3 = (C.c_int64 * 3)(8, 8, 8)
    d1 = (C.c_int64 * 1)(8)
    small = (C.c_int64 * 3)(8, 2, 8)  # ny = 2
    buf = (C.c_float * 512)()
    p = C.cast(buf, C.c_void_p)
    vort = L.pc_fd_vorticity_z
    vort.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_int64), C.c_int, C.c_int, C.c_double, C.c_void_p,
                     C.c_void_p]
    sec = L.pc_fd_second
    sec.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.c_int, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p]
    assert vort(p, p, d1, 1, 1, 1.0, p, None) == 1  # v_x - u_y needs two dimensions
    assert vort(p, p, small, 3, 1, 1.0, p, None) == 1  # and three points along y
    assert vort(p, p, d3, 3, 1, 0.0, p, None) == 1  # h must be positive
    assert vort(p, p, d3, 3, 1, float("nan"), p, None) == 1
    assert vort(p, p, d3, 3, 3, 1.0, p, None) == 1  # bad dtype
    assert vort(p, p, d3, 3, 1, 1.0, p, None) == 1  # host memory
    assert sec(p, d3, 3, 1, 3, 1.0, p, None) == 1  # axis beyond the field
    assert sec(p, (C.c_int64 * 3)(8, 8, 3), 3, 1, 2, 1.0, p, None) == 1  # 3 points along z
    assert sec(p, d3, 0, 1, 0, 1.0, p, None) == 1  # ndims
    assert b"" != L.pc_last_error()
