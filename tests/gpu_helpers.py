"""Test-side helpers for the GPU tests: reading the serialized stream layout
documented in include/pcz.h (pc_streams_serialize) back into numpy arrays."""
import struct

import numpy as np


def parse_serialized(data: bytes):
    """Returns dict(dtype, ndims, dims, n, nbricks, nchunks, comps=[{tau, words,
    counts, measured, chunk_word, brick_len, payload}])."""
    magic, version, dtype, ndims, n, _ = struct.unpack_from("<6I", data, 0)
    dims = struct.unpack_from("<3q", data, 24)
    nbricks, nchunks = struct.unpack_from("<2q", data, 48)
    off = 64
    comps = []
    for i in range(n):
        tau, words = struct.unpack_from("<dQ", data, off)
        counts = list(struct.unpack_from("<5Q", data, off + 16))
        (measured,) = struct.unpack_from("<d", data, off + 56)
        comps.append(dict(tau=tau, words=words, counts=counts, measured=measured))
        off += 64
    for i in range(n):
        c = comps[i]
        c["chunk_word"] = np.frombuffer(data, dtype=np.uint64, count=nchunks, offset=off).copy()
        off += 8 * nchunks
        c["brick_len"] = np.frombuffer(data, dtype=np.uint16, count=nbricks, offset=off).copy()
        off += (2 * nbricks + 7) & ~7
        c["payload"] = np.frombuffer(data, dtype=np.uint64, count=c["words"], offset=off).copy()
        off += 8 * c["words"]
    assert off == len(data)
    return dict(magic=magic, version=version, dtype=dtype, ndims=ndims, dims=dims, n=n, nbricks=nbricks,
                nchunks=nchunks, comps=comps)


def brick_bits(comp, b: int) -> str:
    """The bit string of brick b in a parsed component, as '0'/'1' characters."""
    c = b // 32
    bl = comp["brick_len"].astype(np.int64)
    start = int(comp["chunk_word"][c]) * 64 + int(bl[32 * c:b].sum())
    pl = comp["payload"]
    return "".join(str((int(pl[(start + t) >> 6]) >> ((start + t) & 63)) & 1) for t in range(int(bl[b])))
