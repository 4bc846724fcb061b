"""The debug build (libpcz_debug.so, PCZ_DEBUG): every shared-memory bit write
of the coders and every plane slot and spill index of the retrieval is
checked against its buffer (compute-sanitizer is not available on the GPU
pool, so the library checks itself; a failed check skips the access instead of
faulting).  A child process loads the debug library, runs the coders on 1D,
2D and 3D fields of both types, a batch, served queries and corrupt streams,
checks its results against the oracle, and must end with a clean check word."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
import oracle as O, synth_fields as S
import paper_2308_11759_gb300 as P
assert P.LIBPATH.endswith("libpcz_debug.so"), P.LIBPATH
w, en = P.debug_status(reset=True)
assert en, "not a debug build"
cases = [((37, 29, 41), np.float32, 8), ((21, 19, 17), np.float64, 12), ((130, 97), np.float32, 8),
         ((70, 51), np.float64, 8), ((999,), np.float32, 6), ((1, 1, 1), np.float64, 3)]
for shape, dt, n in cases:
    x = np.ascontiguousarray(S.powerlaw(shape, seed=5, dtype=dt)) if np.prod(shape) > 1 else np.ones(shape, dt)
    tau = O.tau_decade(O.value_range(x) or 1.0, n)
    st = P.compress(torch.from_numpy(x).cuda(), tau)
    ref = O.Streams(x, tau, nthreads=4)
    for k in (1, n // 2, n):
        got = st.retrieve(k=k).cpu().numpy()
        assert np.array_equal(got.view(np.uint8), ref.retrieve(k).view(np.uint8)), (shape, k)
    blob = bytearray(st.serialize())
    blob[-3] ^= 0x5A
    try:
        P.Streams.deserialize(bytes(blob))
    except P.PczError:
        pass
shapes = [(33, 20, 18), (90, 70), (300,)]
plan = P.Batch(shapes, np.float32, 4)
xs = [torch.from_numpy(np.ascontiguousarray(S.powerlaw(s, seed=6, dtype=np.float32))).cuda() for s in shapes]
sts = plan.compress(xs, [P.field_tau_schedule(x, "decade", 4) for x in xs])
P.retrieve_batch(sts, [4] * 3)
srv = P.Server(4 << 30, max_batch=64)
fid = srv.add_field(sts[0])
qs = [(fid, ([4 * (j % 4), 0, 4], [4 * (j % 4) + 12, 16, 16]), 0.0, 1 + j % 4) for j in range(40)]
srv.replay(qs, [0.0] * len(qs))
torch.cuda.synchronize()
w, en = P.debug_status()
print("check word", w)
assert w == 0, hex(w)
'''


def test_debug_build_checks_stay_clean():
    from paper_2308_11759_gb300 import build as B

    B.build(debug=True)
    env = dict(os.environ, PCZ_LIBRARY=B.LIB_DEBUG, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], capture_output=True, text=True, env=env, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "check word 0" in r.stdout
