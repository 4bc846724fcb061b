"""The TMA-staged form of the 3D construction kernel (selected by
PCZ_COMPRESS_TMA=1 when the library is first used; the default form loads the
field with vector loads): in a child process with the variable set, the
streams and reconstructions of fields that take each staging layout (one
128x4x4 box per chunk, one 4x4x4 box per brick with ragged edges) and of one
that falls back to vector loads (rows not a multiple of 16 bytes) equal the
oracle's bit for bit."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import oracle as O
import paper_2308_11759_gb300 as P
import synth_fields as S
from tests.gpu_helpers import parse_serialized

cases = [
    ("row boxes, 128^3 float32", S.powerlaw((128, 128, 128), seed=2, dtype=np.float32), "dec", 4),
    ("brick boxes, 64^3 float64", S.gaussians((64, 64, 64), seed=1), "bin", 4),
    ("brick boxes, ragged 50x42x36 float64", S.powerlaw((50, 42, 36), seed=3, dtype=np.float64), "dec", 6),
    ("vector loads, 45x38x33 float32", S.powerlaw((45, 38, 33), seed=2, dtype=np.float32), "dec", 8),
]
for name, x, kind, n in cases:
    r = O.value_range(x)
    tau = O.tau_decade(r, n) if kind == "dec" else O.tau_binary(r, 4, n)
    xd = torch.from_numpy(x).cuda()
    st = P.compress(xd, tau)
    ref = O.Streams(x, tau, nthreads=8)
    d = parse_serialized(st.serialize())
    for i in range(n):
        c = d["comps"][i]
        assert np.array_equal(c["brick_len"], ref.brick_len(i)), (name, i)
        assert np.array_equal(c["payload"], ref.payload(i)), (name, i)
        assert c["counts"] == [int(v) for v in ref.stats(i)], (name, i)
    got = st.retrieve(k=n).cpu().numpy()
    assert np.array_equal(got.view(np.uint8), ref.retrieve(n).view(np.uint8)), name
    print("ok", name)
"""


def test_tma_staged_construction_equals_oracle():
    env = dict(os.environ, PCZ_COMPRESS_TMA="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("ok ") == 4
