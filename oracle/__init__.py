"""ctypes front end of the CPU oracle (pcz_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the CPU-baseline leg of bench.py.  The product package never imports it.

Arrays follow the field convention of the oracle: a numpy array of shape
(nz, ny, nx) (or (ny, nx), (nx,)) in C order, so dims = shape reversed and x
is the fastest axis.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

F32, F64 = 1, 2
ST_ZERO, ST_CODED, ST_RAW, ST_ESC, ST_VIOL = range(5)

_lib = None


def lib():
    """Loads (building first if needed) liboracle_pcz.so."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        i64p = C.POINTER(C.c_int64)
        u64p = C.POINTER(C.c_uint64)
        dp = C.POINTER(C.c_double)
        vp = C.c_void_p
        sig = {
            "oc_compress": (vp, [vp, C.c_int, C.c_int, i64p, dp, C.c_int, C.c_int]),
            "oc_status": (C.c_int, [vp]),
            "oc_n": (C.c_int, [vp]),
            "oc_nbricks": (C.c_int64, [vp]),
            "oc_nchunks": (C.c_int64, [vp]),
            "oc_payload_words": (C.c_int64, [vp, C.c_int]),
            "oc_payload": (u64p, [vp, C.c_int]),
            "oc_chunk_word": (u64p, [vp, C.c_int]),
            "oc_brick_len": (C.POINTER(C.c_uint16), [vp, C.c_int]),
            "oc_stats": (None, [vp, C.c_int, i64p]),
            "oc_measured": (C.c_double, [vp, C.c_int]),
            "oc_final_xt": (None, [vp, vp]),
            "oc_retrieve": (C.c_int, [vp, C.c_int, C.c_int, i64p, i64p, vp]),
            "oc_free": (None, [vp]),
            "oc_code_brick": (C.c_int, [vp, C.c_int, C.c_int, i64p, dp, C.c_int, C.c_int64, u64p,
                                        C.c_int64, i64p, dp, i64p]),
            "oc_decode_brick": (C.c_int, [C.c_int, C.c_int, dp, C.c_int, u64p, C.c_int64, i64p, dp]),
            "oc_lift_fwd4": (None, [i64p, C.c_int, C.c_int]),
            "oc_lift_inv4": (None, [i64p, C.c_int, C.c_int]),
            "oc_lift_fwd_block": (None, [i64p, C.c_int, C.c_int]),
            "oc_lift_inv_block": (None, [i64p, C.c_int, C.c_int]),
            "oc_perm": (None, [C.c_int, C.POINTER(C.c_int)]),
            "oc_nb_fwd": (C.c_uint64, [C.c_int64, C.c_int]),
            "oc_nb_inv": (C.c_int64, [C.c_uint64, C.c_int]),
            "oc_encode_planes": (C.c_int64, [u64p, C.c_int, C.c_int, C.c_int, u64p, C.c_int64]),
            "oc_decode_planes": (C.c_int64, [u64p, C.c_int64, C.c_int, C.c_int, C.c_int, u64p]),
            "oc_block_emax": (C.c_int, [dp, C.c_int, C.c_int]),
            "oc_quantize": (C.c_int64, [C.c_double, C.c_int]),
            "oc_dequantize": (C.c_double, [C.c_int64, C.c_int, C.c_int]),
            "oc_floor_log2": (C.c_int, [C.c_double]),
            "oc_query_k": (C.c_int, [dp, C.c_int, C.c_double]),
            "oc_gather_brick": (None, [vp, C.c_int, C.c_int, i64p, C.c_int64, dp]),
            "oc_scalar_fl32": (None, [dp, C.c_int64, C.c_int, dp]),
            "oc_version": (C.c_int, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def dtype_code(dt) -> int:
    dt = np.dtype(dt)
    if dt == np.float32:
        return F32
    if dt == np.float64:
        return F64
    raise TypeError(f"unsupported dtype {dt}")


def dims_of(x: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.array(x.shape[::-1], dtype=np.int64))


class Streams:
    """Result of Algorithm 1 on a field: n component streams plus the index."""

    def __init__(self, x: np.ndarray, tau, nthreads: int = 1):
        x = np.ascontiguousarray(x)
        if x.ndim < 1 or x.ndim > 3:
            raise ValueError("1 to 3 dimensions")
        self.x = x
        self.dtype = x.dtype
        self.shape = x.shape
        self.tau = np.ascontiguousarray(np.asarray(tau, dtype=np.float64))
        self.n = len(self.tau)
        self._dims = dims_of(x)
        L = lib()
        self._h = L.oc_compress(x.ctypes.data, dtype_code(x.dtype), x.ndim, _p(self._dims, C.c_int64),
                                _p(self.tau, C.c_double), self.n, nthreads)
        if not self._h:
            raise ValueError("oracle refused the input (bad tau, dims or non-finite values)")
        if L.oc_status(self._h) != 0:
            raise RuntimeError(f"oracle internal failure {L.oc_status(self._h)}")
        self.nbricks = L.oc_nbricks(self._h)
        self.nchunks = L.oc_nchunks(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oc_free(h)
            self._h = None

    def payload(self, i: int) -> np.ndarray:
        L = lib()
        nw = L.oc_payload_words(self._h, i)
        return np.ctypeslib.as_array(L.oc_payload(self._h, i), shape=(max(nw, 1),))[:nw].copy()

    def chunk_word(self, i: int) -> np.ndarray:
        L = lib()
        return np.ctypeslib.as_array(L.oc_chunk_word(self._h, i), shape=(self.nchunks,)).copy()

    def brick_len(self, i: int) -> np.ndarray:
        L = lib()
        return np.ctypeslib.as_array(L.oc_brick_len(self._h, i), shape=(self.nbricks,)).copy()

    def measured(self, i: int) -> float:
        """Computed tolerance of component i+1 (Sec. 4.3): max over the field of
        |fl_T(x - x~_{i+1})|."""
        return float(lib().oc_measured(self._h, i))

    def stats(self, i: int) -> np.ndarray:
        out = np.zeros(5, dtype=np.int64)
        lib().oc_stats(self._h, i, _p(out, C.c_int64))
        return out

    def final_xt(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=self.dtype)
        lib().oc_final_xt(self._h, out.ctypes.data)
        return out

    def retrieve(self, k: int, box=None, k0: int = 0, inout=None) -> np.ndarray:
        """Algorithm 2 with k components (continued from k0 when inout holds x~_k0).

        box = (lo, hi) in array-axis order (z, y, x), half-open."""
        if box is None:
            lo = np.zeros(len(self.shape), dtype=np.int64)
            hi = np.array(self.shape, dtype=np.int64)
        else:
            lo = np.array(box[0], dtype=np.int64)
            hi = np.array(box[1], dtype=np.int64)
        ext = tuple(int(h - l) for l, h in zip(lo, hi))
        lo3 = np.zeros(3, dtype=np.int64)
        hi3 = np.ones(3, dtype=np.int64)
        lo3[: len(ext)] = lo[::-1]
        hi3[: len(ext)] = hi[::-1]
        if inout is None:
            inout = np.zeros(ext, dtype=self.dtype)
        else:
            inout = np.ascontiguousarray(inout, dtype=self.dtype)
        rc = lib().oc_retrieve(self._h, k0, k, _p(lo3, C.c_int64), _p(hi3, C.c_int64), inout.ctypes.data)
        if rc != 0:
            raise RuntimeError("oracle retrieve failed")
        return inout


def code_brick(x: np.ndarray, tau, b: int, maxwords: int = 160):
    """Codes one brick of x for all components; returns (bits[n, maxwords], nbits[n], xt[N], stats[n, 5])."""
    x = np.ascontiguousarray(x)
    tau = np.ascontiguousarray(np.asarray(tau, dtype=np.float64))
    n = len(tau)
    dims = dims_of(x)
    N = 4 ** x.ndim
    bits = np.zeros((n, maxwords), dtype=np.uint64)
    nbits = np.zeros(n, dtype=np.int64)
    xt = np.zeros(N, dtype=np.float64)
    st = np.zeros((n, 5), dtype=np.int64)
    rc = lib().oc_code_brick(x.ctypes.data, dtype_code(x.dtype), x.ndim, _p(dims, C.c_int64),
                             _p(tau, C.c_double), n, int(b), _p(bits, C.c_uint64), maxwords,
                             _p(nbits, C.c_int64), _p(xt, C.c_double), _p(st, C.c_int64))
    if rc != 0:
        raise RuntimeError(f"oracle code_brick failed ({rc})")
    return bits, nbits, xt, st


def decode_brick(dtype, d: int, tau, k: int, bits: np.ndarray, nbits: np.ndarray) -> np.ndarray:
    tau = np.ascontiguousarray(np.asarray(tau, dtype=np.float64))
    bits = np.ascontiguousarray(bits, dtype=np.uint64)
    nbits = np.ascontiguousarray(nbits, dtype=np.int64)
    xt = np.zeros(4 ** d, dtype=np.float64)
    rc = lib().oc_decode_brick(dtype_code(dtype), d, _p(tau, C.c_double), k, _p(bits, C.c_uint64),
                               bits.shape[1], _p(nbits, C.c_int64), _p(xt, C.c_double))
    if rc != 0:
        raise RuntimeError("oracle decode_brick failed")
    return xt


# ---- unit-level entry points used by the pins -------------------------------

def lift_fwd4(v, P):
    a = np.ascontiguousarray(np.array(v, dtype=np.int64))
    lib().oc_lift_fwd4(_p(a, C.c_int64), 1, P)
    return a


def lift_inv4(v, P):
    a = np.ascontiguousarray(np.array(v, dtype=np.int64))
    lib().oc_lift_inv4(_p(a, C.c_int64), 1, P)
    return a


def lift_fwd_block(v, d, P):
    a = np.ascontiguousarray(np.array(v, dtype=np.int64).reshape(-1))
    lib().oc_lift_fwd_block(_p(a, C.c_int64), d, P)
    return a


def lift_inv_block(v, d, P):
    a = np.ascontiguousarray(np.array(v, dtype=np.int64).reshape(-1))
    lib().oc_lift_inv_block(_p(a, C.c_int64), d, P)
    return a


def perm(d):
    N = 4 ** d
    a = np.zeros(N, dtype=np.int32)
    lib().oc_perm(d, _p(a, C.c_int))
    return a


def nb_fwd(q, P):
    return int(lib().oc_nb_fwd(int(q), P))


def nb_inv(u, P):
    return int(lib().oc_nb_inv(int(u), P))


def encode_planes(u, N, P, pmin, maxbits=1 << 14):
    ua = np.ascontiguousarray(np.array(u, dtype=np.uint64))
    out = np.zeros((maxbits + 63) // 64, dtype=np.uint64)
    nb = lib().oc_encode_planes(_p(ua, C.c_uint64), N, P, pmin, _p(out, C.c_uint64), maxbits)
    if nb < 0:
        raise ValueError("too many bits")
    return out, int(nb)


def bits_to_str(words, nbits) -> str:
    return "".join(str((int(words[b >> 6]) >> (b & 63)) & 1) for b in range(nbits))


def str_to_bits(s: str):
    words = np.zeros(max(1, (len(s) + 63) // 64), dtype=np.uint64)
    for b, ch in enumerate(s):
        if ch == "1":
            words[b >> 6] |= np.uint64(1) << np.uint64(b & 63)
    return words, len(s)


def decode_planes(words, nbits, N, P, pmin):
    wa = np.ascontiguousarray(np.array(words, dtype=np.uint64))
    u = np.zeros(N, dtype=np.uint64)
    used = lib().oc_decode_planes(_p(wa, C.c_uint64), nbits, N, P, pmin, _p(u, C.c_uint64))
    return u, int(used)


def block_emax(e, dtype):
    a = np.ascontiguousarray(np.array(e, dtype=np.float64))
    return int(lib().oc_block_emax(_p(a, C.c_double), len(a), dtype_code(dtype)))


def quantize(e, s):
    return int(lib().oc_quantize(float(e), int(s)))


def dequantize(q, s, dtype):
    return float(lib().oc_dequantize(int(q), int(s), dtype_code(dtype)))


def floor_log2(t):
    return int(lib().oc_floor_log2(float(t)))


def query_k(tau, t):
    a = np.ascontiguousarray(np.asarray(tau, dtype=np.float64))
    return int(lib().oc_query_k(_p(a, C.c_double), len(a), float(t)))


def gather_brick(x, b):
    x = np.ascontiguousarray(x)
    dims = dims_of(x)
    out = np.zeros(4 ** x.ndim, dtype=np.float64)
    lib().oc_gather_brick(x.ctypes.data, dtype_code(x.dtype), x.ndim, _p(dims, C.c_int64), int(b),
                          _p(out, C.c_double))
    return out


def scalar_fl32(x, n):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))
    out = np.zeros((n, len(a)), dtype=np.float64)
    lib().oc_scalar_fl32(_p(a, C.c_double), len(a), n, _p(out, C.c_double))
    return out


# ---- tolerance schedules (Sec. 5.1), the oracle side's own copy --------------

def value_range(x) -> float:
    """tau_0 = the range of the field values, max - min, in double."""
    x = np.asarray(x)
    return float(np.float64(x.max()) - np.float64(x.min()))


def tau_binary(rng: float, delta: int, n: int):
    """tau_i = 2^(-delta * i) * tau_0, i = 1..n (exact power-of-two scaling)."""
    return [rng * 2.0 ** (-delta * i) for i in range(1, n + 1)]


def tau_decade(rng: float, n: int, first_exp: int = 2):
    """tau_i = 10^-(first_exp + i - 1) * tau_0, i = 1..n, with each decimal
    factor the double nearest to it and one rounded product."""
    return [float("1e-%d" % (first_exp + i - 1)) * rng for i in range(1, n + 1)]


def bits_as_int(words, nbits) -> int:
    """A bit string (bit b = bit b%64 of word b/64) as a Python integer."""
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint64))
    return int.from_bytes(w.tobytes(), "little") & ((1 << int(nbits)) - 1)
