"""GB300 (sm_103a) implementation of the multi-component progressive-precision
method of Magri & Lindstrom, "A General Framework for Progressive Data
Compression and Retrieval" (Sec. 4, Algorithms 1 and 2).

This module is a thin ctypes binding over libpcz.so (include/pcz.h): it only
marshals arguments (tensor data pointers, shapes, the current CUDA stream).
Every step of compression and retrieval runs in the library's CUDA kernels;
there is no CPU fallback, and importing a function that needs the library
raises if libpcz.so has not been built.

Arrays use C order with shape (nz, ny, nx) for 3D (x fastest); boxes are
given as (lo, hi) in the same axis order, half-open.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PCZ_LIBRARY selects another in-tree build, e.g. libpcz_debug.so (buffer checks)
LIBPATH = os.environ.get("PCZ_LIBRARY") or os.path.join(_HERE, "libpcz.so")

PC_F32, PC_F64 = 1, 2
STATUS = {
    0: "PC_OK", 1: "PC_ERR_ARG", 2: "PC_ERR_TAU_ORDER", 3: "PC_ERR_NONFINITE", 4: "PC_ERR_OOM",
    5: "PC_ERR_CUDA", 6: "PC_ERR_CORRUPT_STREAM", 7: "PC_ERR_TOL_UNREACHABLE", 8: "PC_ERR_VERSION",
}


class PczError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class Box(C.Structure):
    _fields_ = [("lo", C.c_int64 * 3), ("hi", C.c_int64 * 3)]


class Query(C.Structure):
    _fields_ = [("field", C.c_int), ("k", C.c_int), ("tau", C.c_double), ("box", Box)]


class ServeStats(C.Structure):
    _fields_ = [("wall_s", C.c_double), ("batches", C.c_uint64), ("queries", C.c_uint64),
                ("bytes_out", C.c_uint64), ("max_batch", C.c_uint64), ("peak_device_bytes", C.c_uint64),
                ("arena_bytes", C.c_uint64), ("max_inflight", C.c_uint64)]


PC_SERVE_NO_CACHE, PC_SERVE_SERIAL = 1, 2


class BatchInfo(C.Structure):
    _fields_ = [("schedule", C.c_int), ("order", C.c_int), ("chunks_per_item", C.c_int),
                ("items_per_claim", C.c_int), ("candidates", C.c_int), ("grid", C.c_int), ("graph", C.c_int),
                ("ctas_per_sm", C.c_int), ("warps_small", C.c_int), ("mixed", C.c_int), ("calls", C.c_uint64),
                ("candidate_ms", C.c_double * 16)]


_lib = None


def lib():
    """The loaded libpcz.so (raises if it is missing: no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise ImportError(f"{LIBPATH} is not built; run __graft_entry__.build() (there is no CPU fallback)")
        L = C.CDLL(LIBPATH)
        vp, i64p, dp, ip = C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_int)
        u64p = C.POINTER(C.c_uint64)
        sig = {
            "pc_compress": [vp, i64p, C.c_int, C.c_int, dp, C.c_int, vp, C.POINTER(vp)],
            "pc_query_k": [vp, C.c_double, ip],
            "pc_query_k_measured": [vp, C.c_double, ip],
            "pc_stream_measured_error": [vp, C.c_int, dp],
            "pc_retrieve": [vp, C.c_double, C.c_int, C.POINTER(Box), vp, vp],
            "pc_refine": [vp, C.c_int, C.c_int, C.POINTER(Box), vp, vp],
            "pc_stream_info": [vp, C.c_int, dp, u64p, u64p],
            "pc_streams_shape": [vp, ip, i64p, ip, ip],
            "pc_stream_counts": [vp, C.c_int, u64p],
            "pc_streams_serialize": [vp, vp, C.POINTER(C.c_size_t), vp],
            "pc_streams_deserialize": [vp, C.c_size_t, vp, C.POINTER(vp)],
            "pc_stream_device_ptrs": [vp, C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), u64p, u64p, u64p],
            "pc_field_range": [vp, C.c_int64, C.c_int, vp, dp, dp],
            "pc_stream_read_index": [vp, C.c_int, u64p, C.POINTER(C.c_uint16), vp],
            "pc_stream_read": [vp, C.c_int, C.c_uint64, C.c_uint64, u64p, vp],
            "pc_server_create": [C.c_uint64, C.c_int, C.c_int, vp, C.POINTER(vp)],
            "pc_debug_status": [C.POINTER(C.c_uint32), ip, C.c_int],
            "pc_batch_create": [C.c_int, i64p, ip, C.c_int, C.c_int, vp, C.POINTER(vp)],
            "pc_batch_compress": [vp, C.POINTER(vp), dp, C.POINTER(vp)],
            "pc_batch_info": [vp, C.POINTER(BatchInfo)],
            "pc_batch_free": [vp],
            "pc_retrieve_batch": [C.c_int, C.POINTER(vp), ip, C.POINTER(Box), C.POINTER(vp), vp],
            "pc_server_add_field": [vp, vp, ip],
            "pc_server_replay": [vp, C.POINTER(Query), dp, C.c_int, C.POINTER(vp), dp, C.POINTER(ServeStats)],
            "pc_server_reset_cache": [vp],
            "pc_server_free": [vp],
            "pc_server_submit": [vp, C.POINTER(Query), vp, u64p],
            "pc_server_poll": [vp, C.c_uint64, ip, dp],
            "pc_server_wait": [vp, C.c_uint64, C.c_double, ip, dp],
            "pc_server_stats": [vp, C.POINTER(ServeStats)],
            "pc_tau_schedule": [C.c_int, C.c_double, C.c_int, C.c_int, dp],
            "pc_field_tau_schedule": [vp, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int, vp, dp],
            "pc_lossless_sweep": [vp, i64p, C.c_int, C.c_int, C.c_int, C.c_int, vp, C.POINTER(vp), ip, dp],
            "pc_fd_vorticity_z": [vp, vp, i64p, C.c_int, C.c_int, C.c_double, vp, vp],
            "pc_fd_second": [vp, i64p, C.c_int, C.c_int, C.c_int, C.c_double, vp, vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.pc_timing_enable.argtypes = [C.c_int]
        L.pc_timing_enable.restype = C.c_int
        L.pc_timing_read.argtypes = [C.POINTER(C.c_double), u64p]
        L.pc_timing_read.restype = C.c_int
        L.pc_streams_free.argtypes = [vp]
        L.pc_streams_free.restype = None
        L.pc_last_error.argtypes = []
        L.pc_last_error.restype = C.c_char_p
        L.pc_release_cached_memory.argtypes = []
        L.pc_release_cached_memory.restype = C.c_int
        L.pc_version.argtypes = []
        L.pc_version.restype = C.c_int
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise PczError(status, lib().pc_last_error().decode())


def _torch():
    import torch

    return torch


def _dtype_code(dt) -> int:
    torch = _torch()
    if dt in (torch.float32, np.float32) or str(dt) in ("float32", "torch.float32"):
        return PC_F32
    if dt in (torch.float64, np.float64) or str(dt) in ("float64", "torch.float64"):
        return PC_F64
    raise TypeError(f"unsupported dtype {dt}")


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _box(box, shape):
    if box is None:
        return None, tuple(shape)
    lo, hi = [int(v) for v in box[0]], [int(v) for v in box[1]]
    nd = len(shape)
    if len(lo) != nd or len(hi) != nd:
        raise ValueError("box rank differs from the field's")
    b = Box()
    for a in range(3):
        b.lo[a] = lo[nd - 1 - a] if a < nd else 0
        b.hi[a] = hi[nd - 1 - a] if a < nd else 1
    return b, tuple(h - l for l, h in zip(lo, hi))


def _ptr(x):
    torch = _torch()
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(x.ctypes.data)
    raise TypeError("expected a torch tensor or a numpy array")


class Streams:
    """The n compressed components of one field (Algorithm 1's output)."""

    def __init__(self, handle, shape, dtype):
        self._h = handle
        self.shape = tuple(shape)
        self.dtype = dtype
        n = C.c_int()
        _check(lib().pc_streams_shape(self._h, None, None, None, C.byref(n)))
        self.n = n.value

    # ---- construction ---------------------------------------------------
    @classmethod
    def compress(cls, x, tau, stream=None):
        """Algorithm 1 on x (CUDA tensor, or host tensor/array copied in by the
        library) with tolerances tau (strictly decreasing, > 0)."""
        torch = _torch()
        shape = tuple(x.shape)
        dims = (C.c_int64 * 3)(*([int(s) for s in shape[::-1]] + [1] * (3 - len(shape))))
        taus = (C.c_double * len(tau))(*[float(t) for t in tau])
        h = C.c_void_p()
        dt = x.dtype if isinstance(x, torch.Tensor) else x.dtype.type
        _check(lib().pc_compress(_ptr(x), dims, len(shape), _dtype_code(dt), taus, len(tau), _stream_ptr(stream),
                                 C.byref(h)))
        tdt = x.dtype if isinstance(x, torch.Tensor) else (torch.float32 if x.dtype == np.float32 else torch.float64)
        return cls(h, shape, tdt)

    @classmethod
    def deserialize(cls, data: bytes, stream=None):
        torch = _torch()
        buf = C.create_string_buffer(bytes(data), len(data))
        h = C.c_void_p()
        _check(lib().pc_streams_deserialize(buf, len(data), _stream_ptr(stream), C.byref(h)))
        nd = C.c_int()
        dims = (C.c_int64 * 3)()
        dt = C.c_int()
        _check(lib().pc_streams_shape(h, C.byref(nd), dims, C.byref(dt), None))
        shape = tuple(int(dims[a]) for a in range(nd.value))[::-1]
        return cls(h, shape, torch.float32 if dt.value == PC_F32 else torch.float64)

    def close(self):
        if getattr(self, "_h", None):
            lib().pc_streams_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- queries --------------------------------------------------------
    def query_k(self, tau: float, measured: bool = False) -> int:
        """Components a query at tolerance tau needs: on the prescribed
        tolerances (Sec. 6.2), or on the computed ones (Sec. 4.3)."""
        k = C.c_int()
        fn = lib().pc_query_k_measured if measured else lib().pc_query_k
        _check(fn(self._h, float(tau), C.byref(k)))
        return k.value

    def measured_error(self, i: int) -> float:
        """Computed tolerance of component i+1: max |fl(x - x~_{i+1})| (Sec. 4.3)."""
        e = C.c_double()
        _check(lib().pc_stream_measured_error(self._h, i, C.byref(e)))
        return e.value

    def tau(self, i: int) -> float:
        t = C.c_double()
        _check(lib().pc_stream_info(self._h, i, C.byref(t), None, None))
        return t.value

    def info(self, i: int):
        t, bits, idx = C.c_double(), C.c_uint64(), C.c_uint64()
        _check(lib().pc_stream_info(self._h, i, C.byref(t), C.byref(bits), C.byref(idx)))
        return t.value, bits.value, idx.value

    def counts(self, i: int):
        out = (C.c_uint64 * 5)()
        _check(lib().pc_stream_counts(self._h, i, out))
        return [int(v) for v in out]

    def device_ptrs(self, i: int):
        pl, cw, bl = C.c_void_p(), C.c_void_p(), C.c_void_p()
        nw, nc, nb = C.c_uint64(), C.c_uint64(), C.c_uint64()
        _check(lib().pc_stream_device_ptrs(self._h, i, C.byref(pl), C.byref(cw), C.byref(bl), C.byref(nw),
                                           C.byref(nc), C.byref(nb)))
        return pl.value, cw.value, bl.value, nw.value, nc.value, nb.value

    # ---- reconstruction -------------------------------------------------
    def retrieve(self, k=None, tau=None, box=None, out=None, stream=None):
        """Algorithm 2: x~_k on the box (k given, or the smallest k meeting tau).
        Writes into out (device or host tensor/array) or a new CUDA tensor."""
        torch = _torch()
        b, ext = _box(box, self.shape)
        if out is None:
            out = torch.empty(ext, dtype=self.dtype, device="cuda")
        t = -1.0 if tau is None else float(tau)
        kk = 0 if k is None else int(k)
        if tau is None and k is None:
            raise ValueError("give k or tau")
        _check(lib().pc_retrieve(self._h, t, kk, C.byref(b) if b is not None else None, _ptr(out),
                                 _stream_ptr(stream)))
        return out

    def refine(self, k0: int, k: int, inout, box=None, stream=None):
        """Adds components k0+1..k into inout, which holds x~_k0 on the box."""
        b, _ = _box(box, self.shape)
        _check(lib().pc_refine(self._h, int(k0), int(k), C.byref(b) if b is not None else None, _ptr(inout),
                               _stream_ptr(stream)))
        return inout

    def read_index(self, i: int, stream=None):
        """(chunk_word[nchunks] u64, brick_len[nbricks] u16) of component i, on the host."""
        _, _, _, _, nc, nb = self.device_ptrs(i)
        cw = np.zeros(nc, dtype=np.uint64)
        bl = np.zeros(nb, dtype=np.uint16)
        _check(lib().pc_stream_read_index(self._h, i, cw.ctypes.data_as(C.POINTER(C.c_uint64)),
                                          bl.ctypes.data_as(C.POINTER(C.c_uint16)), _stream_ptr(stream)))
        return cw, bl

    def read_payload(self, i: int, word_off: int, nwords: int, stream=None) -> np.ndarray:
        out = np.zeros(max(nwords, 1), dtype=np.uint64)
        _check(lib().pc_stream_read(self._h, i, int(word_off), int(nwords), out.ctypes.data_as(C.POINTER(C.c_uint64)),
                                    _stream_ptr(stream)))
        return out[:nwords]

    def brick_bits(self, i: int, b: int, index=None):
        """Brick b's bit string in component i as (python int, bit length)."""
        cw, bl = index if index is not None else self.read_index(i)
        c = b // 32
        start = int(cw[c]) * 64 + int(bl[32 * c:b].astype(np.int64).sum())
        nbits = int(bl[b])
        w0 = start // 64
        nw = (start + nbits + 63) // 64 - w0
        words = self.read_payload(i, w0, nw)
        v = int.from_bytes(words.tobytes(), "little") >> (start - 64 * w0)
        return v & ((1 << nbits) - 1), nbits

    def serialize(self, stream=None) -> bytes:
        n = C.c_size_t()
        _check(lib().pc_streams_serialize(self._h, None, C.byref(n), _stream_ptr(stream)))
        buf = C.create_string_buffer(n.value)
        _check(lib().pc_streams_serialize(self._h, buf, C.byref(n), _stream_ptr(stream)))
        return buf.raw[: n.value]


class Batch:
    """A plan for compressing many fields of fixed shapes at once (pc_batch_*):
    one persistent launch over all fields' chunks, replayed as a CUDA graph,
    schedule picked by an autotuner on the first call."""

    def __init__(self, shapes, dtype, n: int, stream=None):
        self.shapes = [tuple(int(v) for v in sh) for sh in shapes]
        self.dtype = dtype
        self.n = int(n)
        nf = len(self.shapes)
        dims = (C.c_int64 * (3 * nf))()
        nds = (C.c_int * nf)()
        for f, sh in enumerate(self.shapes):
            rev = list(sh[::-1]) + [1] * (3 - len(sh))
            for a in range(3):
                dims[3 * f + a] = rev[a]
            nds[f] = len(sh)
        self._h = C.c_void_p()
        _check(lib().pc_batch_create(nf, dims, nds, _dtype_code(dtype), self.n, _stream_ptr(stream),
                                     C.byref(self._h)))

    def compress(self, fields, taus):
        """fields: CUDA tensors of the plan's shapes; taus: one list of n
        tolerances per field.  Returns one Streams per field."""
        nf = len(self.shapes)
        if len(fields) != nf or len(taus) != nf:
            raise ValueError("one field and one tolerance list per planned shape")
        for x, sh in zip(fields, self.shapes):
            if tuple(x.shape) != sh:
                raise ValueError(f"field of shape {tuple(x.shape)} where {sh} was planned")
        ptrs = (C.c_void_p * nf)(*[_ptr(x).value for x in fields])
        flat = [float(t) for tl in taus for t in tl]
        if len(flat) != nf * self.n:
            raise ValueError("n tolerances per field")
        tau = (C.c_double * len(flat))(*flat)
        outs = (C.c_void_p * nf)()
        _check(lib().pc_batch_compress(self._h, ptrs, tau, outs))
        torch = _torch()
        tdt = torch.float32 if _dtype_code(self.dtype) == PC_F32 else torch.float64
        return [Streams(C.c_void_p(outs[f]), self.shapes[f], tdt) for f in range(nf)]

    def info(self):
        inf = BatchInfo()
        _check(lib().pc_batch_info(self._h, C.byref(inf)))
        d = {name: getattr(inf, name) for name, _ in BatchInfo._fields_ if name != "candidate_ms"}
        d["candidate_ms"] = [inf.candidate_ms[i] for i in range(inf.candidates)]
        return d

    def close(self):
        if self._h:
            lib().pc_batch_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def retrieve_batch(streams, ks, boxes=None, outs=None, stream=None):
    """Algorithm 2 for many (streams, k, box) queries in one launch per type
    and dimensionality (pc_retrieve_batch).  Returns the output tensors."""
    torch = _torch()
    nq = len(streams)
    bx = (Box * max(nq, 1))()
    res = []
    for q in range(nq):
        st = streams[q]
        box = boxes[q] if boxes is not None else None
        b, ext = _box(box, st.shape)
        if b is None:
            b, ext = _box(([0] * len(st.shape), list(st.shape)), st.shape)
        bx[q] = b
        res.append(outs[q] if outs is not None else torch.empty(ext, dtype=st.dtype, device="cuda"))
    sp = (C.c_void_p * max(nq, 1))(*[st._h.value for st in streams])
    kk = (C.c_int * max(nq, 1))(*[int(k) for k in ks])
    op = (C.c_void_p * max(nq, 1))(*[o.data_ptr() for o in res])
    _check(lib().pc_retrieve_batch(nq, sp, kk, bx, op, _stream_ptr(stream)))
    return res


class Server:
    """Progressive-query server over device-resident streams (pc_server_*):
    batched retrieval with a per-field cache of partial sums, admission by a
    device-memory budget."""

    def __init__(self, budget_bytes: int, max_batch: int = 256, cache: bool = True, serial: bool = False,
                 stream=None):
        flags = (0 if cache else PC_SERVE_NO_CACHE) | (PC_SERVE_SERIAL if serial else 0)
        self._h = C.c_void_p()
        self._fields = []  # keeps the Streams objects alive
        _check(lib().pc_server_create(int(budget_bytes), int(max_batch), flags, _stream_ptr(stream),
                                      C.byref(self._h)))

    def add_field(self, streams: "Streams") -> int:
        fid = C.c_int()
        _check(lib().pc_server_add_field(self._h, streams._h, C.byref(fid)))
        self._fields.append(streams)
        return fid.value

    def replay(self, queries, arrival_s, outs=None):
        """queries: list of (field, box, tau, k) with box = (lo, hi) in array
        axis order (k = 0: take k from tau); arrival_s: non-decreasing
        seconds.  outs: optional list of CUDA tensors (or None) receiving the
        results.  Returns (latencies in seconds as a numpy array, stats dict)."""
        nq = len(queries)
        qa = (Query * max(nq, 1))()
        for j, (field, box, tau, k) in enumerate(queries):
            known = 0 <= field < len(self._fields)  # the library rejects other indices
            shape = self._fields[field].shape if known else tuple(box[1])
            b, _ = _box(box, shape)
            qa[j].field = int(field)
            qa[j].k = int(k)
            qa[j].tau = float(tau)
            qa[j].box = b if b is not None else _box(([0] * len(shape), list(shape)), shape)[0]
        arr = (C.c_double * max(nq, 1))(*[float(t) for t in arrival_s])
        lat = (C.c_double * max(nq, 1))()
        outp = None
        if outs is not None:
            outp = (C.c_void_p * max(nq, 1))(*[(o.data_ptr() if o is not None else None) for o in outs])
        st = ServeStats()
        _check(lib().pc_server_replay(self._h, qa, arr, nq, outp, lat, C.byref(st)))
        stats = {name: getattr(st, name) for name, _ in ServeStats._fields_}
        return np.frombuffer(lat, dtype=np.float64, count=nq).copy(), stats

    def _query(self, field, box, tau, k):
        known = 0 <= field < len(self._fields)  # the library rejects other indices
        shape = self._fields[field].shape if known else tuple(box[1])
        b, _ = _box(box, shape)
        q = Query()
        q.field = int(field)
        q.k = int(k)
        q.tau = float(tau)
        q.box = b if b is not None else _box(([0] * len(shape), list(shape)), shape)[0]
        return q

    def submit(self, field, box, tau=0.0, k=0, out=None) -> int:
        """Online: queues one query (k = 0: k from tau) and returns its ticket at
        once; out (a CUDA tensor of the box's shape, or None) receives the result."""
        t = C.c_uint64()
        q = self._query(field, box, tau, k)
        _check(lib().pc_server_submit(self._h, C.byref(q), _ptr(out) if out is not None else None, C.byref(t)))
        return t.value

    def poll(self, ticket: int):
        """(done, latency in seconds or None) without blocking."""
        d, lat = C.c_int(), C.c_double()
        _check(lib().pc_server_poll(self._h, int(ticket), C.byref(d), C.byref(lat)))
        return bool(d.value), (lat.value if d.value else None)

    def wait(self, ticket: int, timeout_s: float = -1.0):
        """Blocks until the query is done (or the timeout passes); (done, latency)."""
        d, lat = C.c_int(), C.c_double()
        _check(lib().pc_server_wait(self._h, int(ticket), float(timeout_s), C.byref(d), C.byref(lat)))
        return bool(d.value), (lat.value if d.value else None)

    def stats(self):
        st = ServeStats()
        _check(lib().pc_server_stats(self._h, C.byref(st)))
        return {name: getattr(st, name) for name, _ in ServeStats._fields_}

    def reset_cache(self):
        _check(lib().pc_server_reset_cache(self._h))

    def close(self):
        if self._h:
            lib().pc_server_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def compress(x, tau, stream=None) -> Streams:
    return Streams.compress(x, tau, stream)


def field_range(x, stream=None):
    """(min, max) of a CUDA tensor, reduced on the device."""
    lo, hi = C.c_double(), C.c_double()
    _check(lib().pc_field_range(_ptr(x), x.numel(), _dtype_code(x.dtype), _stream_ptr(stream), C.byref(lo),
                                C.byref(hi)))
    return lo.value, hi.value


# ---- derivatives of reconstructions (Sec. 5.3, the progressive use case) ----


def _fd_out(x, out):
    torch = _torch()
    if out is None:
        out = torch.empty_like(x)
    if out.shape != x.shape or out.dtype != x.dtype:
        raise ValueError("out must have the input's shape and type")
    return out


def fd_vorticity_z(u, v, h: float = 1.0, out=None, stream=None):
    """omega_z = v_x - u_y of device tensors u, v of shape (nz, ny, nx) or
    (ny, nx), grid spacing h (pc_fd_vorticity_z)."""
    if u.shape != v.shape or u.dtype != v.dtype:
        raise ValueError("u and v must have one shape and one type")
    out = _fd_out(u, out)
    dims = (C.c_int64 * u.dim())(*reversed(u.shape))
    _check(lib().pc_fd_vorticity_z(_ptr(u), _ptr(v), dims, u.dim(), _dtype_code(u.dtype), float(h), _ptr(out),
                                   _stream_ptr(stream)))
    return out


def fd_second(w, axis: int, h: float = 1.0, out=None, stream=None):
    """The second derivative of device tensor w along grid axis `axis` (0 = x,
    the last tensor dimension), grid spacing h (pc_fd_second)."""
    out = _fd_out(w, out)
    dims = (C.c_int64 * w.dim())(*reversed(w.shape))
    _check(lib().pc_fd_second(_ptr(w), dims, w.dim(), _dtype_code(w.dtype), int(axis), float(h), _ptr(out),
                              _stream_ptr(stream)))
    return out


# ---- tolerance schedules (Sec. 5.1: tau_i = 2^(-delta i) tau_0, tau_0 = range) ----

PC_TAU_BINARY, PC_TAU_DECADE = 1, 2


def _schedule(kind, tau0, param, n):
    out = (C.c_double * n)()
    _check(lib().pc_tau_schedule(kind, float(tau0), int(param), int(n), out))
    return list(out)


def tau_binary(tau0: float, delta: int, n: int):
    """tau_i = 2^(-delta * i) * tau_0 for i = 1..n (pc_tau_schedule)."""
    return _schedule(PC_TAU_BINARY, tau0, delta, n)


def tau_decade(tau0: float, n: int, first_exp: int = 2):
    """tau_i = 10^-(first_exp + i - 1) * tau_0 for i = 1..n (pc_tau_schedule)."""
    return _schedule(PC_TAU_DECADE, tau0, first_exp, n)


def field_tau_schedule(x, kind: str, n: int, param=None, stream=None):
    """The schedule of a CUDA tensor (or pinned host tensor) relative to its own
    range, tau_0 = max - min reduced on the device (pc_field_tau_schedule):
    kind "binary" (param = delta, default 4) or "decade" (param = first
    exponent, default 2)."""
    code = {"binary": PC_TAU_BINARY, "decade": PC_TAU_DECADE}[kind]
    if param is None:
        param = 4 if kind == "binary" else 2
    out = (C.c_double * n)()
    _check(lib().pc_field_tau_schedule(_ptr(x), x.numel(), _dtype_code(x.dtype), code, int(param), int(n),
                                       _stream_ptr(stream), out))
    return list(out)


def lossless_sweep(x, delta: int = 4, n_max: int = 64, stream=None):
    """Sec. 5.1.3 (pc_lossless_sweep): components are added until x~ reproduces
    x, with the binary schedule tau_i = 2^(-delta i) * range.  Returns dict(k =
    the first component whose computed tolerance is 0 (None if none),
    bits_per_value = stream bits of components 1..k including their index,
    ratio = bits of the type / bits_per_value, measured = the computed
    tolerances, streams = the Streams object)."""
    dims = (C.c_int64 * 3)(*([int(v) for v in reversed(x.shape)] + [1] * (3 - x.dim())))
    h = C.c_void_p()
    k = C.c_int()
    bpv = C.c_double()
    _check(lib().pc_lossless_sweep(_ptr(x), dims, x.dim(), _dtype_code(x.dtype), int(delta), int(n_max),
                                   _stream_ptr(stream), C.byref(h), C.byref(k), C.byref(bpv)))
    st = Streams(h, tuple(x.shape), x.dtype)
    meas = [st.measured_error(i) for i in range(st.n)]
    tbits = 32 if st.dtype in (_torch().float32,) else 64
    kk = k.value or None
    return {"k": kk, "bits_per_value": bpv.value if kk else None, "ratio": (tbits / bpv.value) if kk else None,
            "measured": meas, "streams": st}


def debug_status(reset: bool = False):
    """(check word, enabled): the buffer-check failures a debug build has seen
    (pc_debug_status); a release build reports (0, False)."""
    w, en = C.c_uint32(), C.c_int()
    _check(lib().pc_debug_status(C.byref(w), C.byref(en), 1 if reset else 0))
    return int(w.value), bool(en.value)


KERNEL_KINDS = ("compress", "scan", "pack", "retrieve", "range", "fd")


def release_cached_memory():
    """Returns the device memory the library keeps for later calls (freed
    streams, scratch, the construction bit pool) to the driver."""
    _check(lib().pc_release_cached_memory())


def timing_enable(on: bool = True):
    """Start (or stop) per-kernel CUDA-event timing inside the library."""
    _check(lib().pc_timing_enable(1 if on else 0))


def timing_read():
    """{kernel kind: (total ms, launches)} since timing_enable."""
    ms = (C.c_double * len(KERNEL_KINDS))()
    n = (C.c_uint64 * len(KERNEL_KINDS))()
    _check(lib().pc_timing_read(ms, n))
    return {k: (ms[i], int(n[i])) for i, k in enumerate(KERNEL_KINDS)}
