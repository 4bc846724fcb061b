"""Batched construction and retrieval (pc_batch_*, pc_retrieve_batch): every
field's streams from one persistent, graph-replayed launch over a mixed batch
of 1D, 2D and 3D fields equal pc_compress's streams for that field alone, bit
for bit (and, for a sample, the oracle's); a second call on the same plan
with new values and tolerances does too; batched retrieval equals per-query
retrieval."""
import numpy as np
import pytest

import oracle as O
import synth_fields as S
from tests.gpu_helpers import parse_serialized

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [(37, 29, 41), (130, 97), (16, 16, 16), (5, 300), (1201,), (9, 13, 70), (64, 64), (3, 3, 3),
          (211, 45), (40, 33, 20), (1, 77), (96, 8, 8)]


@pytest.fixture(scope="module")
def P():
    import paper_2308_11759_gb300 as pcz

    pcz.lib()
    return pcz


def _fields(dtype, seed):
    out = []
    for j, sh in enumerate(SHAPES):
        f = S.gaussians(sh, seed=seed + j) if j % 2 else S.powerlaw(sh, seed=seed + j, dtype=np.float64)
        out.append(np.ascontiguousarray(f.astype(dtype)))
    return out


def _taus(xs, n, first_exp):
    return [O.tau_decade(O.value_range(x), n, first_exp=first_exp) for x in xs]


def _check_equal_alone(P, xs, taus, got, oracle_every=0):
    for j, (x, tau, st) in enumerate(zip(xs, taus, got)):
        alone = P.compress(torch.from_numpy(x).cuda(), tau)
        assert st.serialize() == alone.serialize(), SHAPES[j]
        for i in range(st.n):
            assert st.measured_error(i) == alone.measured_error(i)
        if oracle_every and j % oracle_every == 0:
            ref = O.Streams(x, tau, nthreads=4)
            d = parse_serialized(st.serialize())
            for i in range(ref.n):
                assert np.array_equal(d["comps"][i]["payload"], ref.payload(i))
                assert np.array_equal(d["comps"][i]["brick_len"], ref.brick_len(i))
        alone.close()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_batch_equals_alone_and_replays(P, dtype):
    n = 6
    plan = P.Batch(SHAPES, dtype, n)
    xs = _fields(dtype, 40)
    taus = _taus(xs, n, 2)
    got = plan.compress([torch.from_numpy(x).cuda() for x in xs], taus)
    _check_equal_alone(P, xs, taus, got, oracle_every=3)
    info = plan.info()
    assert info["graph"] == 1 and info["calls"] == 1
    assert 0 <= info["schedule"] < info["candidates"]
    timed = [ms for ms in info["candidate_ms"] if ms != -1.0]
    assert all(ms > 0 for ms in timed)
    # float64 has no 16-warp 1D/2D or mixed schedule (128 registers a thread
    # are too few for a 2D float64 brick): 9 of the 16 schedules remain
    assert len(timed) == (16 if dtype == np.float32 else 9)
    assert info["candidate_ms"][info["schedule"]] > 0
    # the same plan, new values and tolerances: the graph replays with new parameters
    xs2 = _fields(dtype, 90)
    taus2 = _taus(xs2, n, 1)
    got2 = plan.compress([torch.from_numpy(x).cuda() for x in xs2], taus2)
    _check_equal_alone(P, xs2, taus2, got2)
    assert plan.info()["calls"] == 2
    # streams of one batch share device arrays: free them in any order, use the rest
    for st in got[::2]:
        st.close()
    for j in range(1, len(got), 2):
        want = P.compress(torch.from_numpy(xs[j]).cuda(), taus[j]).retrieve(k=3)
        assert torch.equal(got[j].retrieve(k=3).view(torch.uint8), want.view(torch.uint8))
    plan.close()


def test_retrieve_batch_equals_per_query(P):
    n = 6
    xs = _fields(np.float32, 7)
    taus = _taus(xs, n, 2)
    plan = P.Batch(SHAPES, np.float32, n)
    sts = plan.compress([torch.from_numpy(x).cuda() for x in xs], taus)
    rng = np.random.default_rng(12)
    qs, ks, boxes = [], [], []
    for _ in range(60):
        j = int(rng.integers(0, len(SHAPES)))
        sh = SHAPES[j]
        lo = [int(rng.integers(0, s)) for s in sh]
        hi = [int(rng.integers(l + 1, s + 1)) for l, s in zip(lo, sh)]
        qs.append(sts[j])
        ks.append(int(rng.integers(0, n + 1)))
        boxes.append((lo, hi))
    outs = P.retrieve_batch(qs, ks, boxes)
    for st, k, box, o in zip(qs, ks, boxes, outs):
        want = st.retrieve(k=k, box=box)
        assert torch.equal(o.view(torch.uint8), want.view(torch.uint8))
    full = P.retrieve_batch(sts, [n] * len(sts))
    for st, o in zip(sts, full):
        assert torch.equal(o.view(torch.uint8), st.retrieve(k=n).view(torch.uint8))
    plan.close()


def test_batch_errors(P):
    shapes = [(20, 20), (8, 8, 8)]
    plan = P.Batch(shapes, np.float32, 3)
    xs = [np.ascontiguousarray(S.powerlaw(sh, seed=3, dtype=np.float32)) for sh in shapes]
    with pytest.raises(P.PczError) as e:
        plan.compress([torch.from_numpy(x).cuda() for x in xs], [[0.1, 0.2, 0.01], [0.1, 0.01, 0.001]])
    assert e.value.name == "PC_ERR_TAU_ORDER"
    bad = xs[1].copy()
    bad[3, 3, 3] = np.nan
    with pytest.raises(P.PczError) as e:
        plan.compress([torch.from_numpy(xs[0]).cuda(), torch.from_numpy(bad).cuda()],
                      [[0.1, 0.01, 0.001], [0.1, 0.01, 0.001]])
    assert e.value.name == "PC_ERR_NONFINITE"
    with pytest.raises(P.PczError) as e:
        plan.compress([torch.from_numpy(x) for x in xs], [[0.1, 0.01, 0.001]] * 2)  # host tensors
    assert e.value.name == "PC_ERR_ARG"
    # the plan still works after the errors
    sts = plan.compress([torch.from_numpy(x).cuda() for x in xs], [[0.1, 0.01, 0.001]] * 2)
    for x, st in zip(xs, sts):
        assert st.serialize() == P.compress(torch.from_numpy(x).cuda(), [0.1, 0.01, 0.001]).serialize()
    plan.close()
