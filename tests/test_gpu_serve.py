"""Progressive-query server (pc_server_*): every result of a batched,
cached, memory-admitted request stream equals the same query run alone
through pc_retrieve, bit for bit, and a sample equals the oracle's x~_k on the
box.  The same holds with the cache off, in the unbatched serial mode, on a
warm cache, and under a budget that forces queries to wait for memory."""
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


@pytest.fixture(scope="module")
def fields(P):
    """Three float32 fields (one ragged) and one float64 field, 8 components each."""
    specs = [((64, 64, 64), 2, np.float32), ((37, 41, 46), 3, np.float32), ((32, 32, 32), 4, np.float32),
             ((24, 28, 20), 5, np.float64)]
    out = []
    for shape, seed, dt in specs:
        x = S.powerlaw(shape, seed=seed, dtype=dt)
        tau = O.tau_decade(O.value_range(x), 8)
        xd = torch.from_numpy(x).cuda()
        out.append((x, xd, tau, P.compress(xd, tau)))
    return out


def _queries(fields, nq, seed, aligned_only=False):
    rng = np.random.default_rng(seed)
    qs = []
    for _ in range(nq):
        f = int(rng.integers(0, len(fields)))
        x, _, tau, _ = fields[f]
        lo, hi = [], []
        for s in x.shape:
            if aligned_only or rng.random() < 0.7:  # brick-aligned origin, side a multiple of 4
                nbk = (s + 3) // 4
                b0 = int(rng.integers(0, nbk))
                side = 4 * int(rng.integers(1, nbk - b0 + 1))
                lo.append(4 * b0)
                hi.append(min(4 * b0 + side, s))
            else:  # arbitrary box
                a = int(rng.integers(0, s))
                lo.append(a)
                hi.append(int(rng.integers(a + 1, s + 1)))
        if rng.random() < 0.5:
            k = int(rng.integers(1, 9))
            qs.append((f, (lo, hi), 0.0, k))
        else:  # by tolerance, log-uniform between tau_8 and tau_1 (relative)
            t = tau[0] * 10.0 ** (-7.0 * rng.random())
            qs.append((f, (lo, hi), t, 0))
    return qs


def _alone(P, fields, q):
    f, box, t, k = q
    st = fields[f][3]
    return st.retrieve(k=k, box=box) if k else st.retrieve(tau=t, box=box)


def _run(P, fields, qs, arrivals, **kw):
    srv = P.Server(kw.pop("budget", 8 << 30), **kw)
    for _, _, _, st in fields:
        srv.add_field(st)
    outs = [torch.empty(tuple(h - l for l, h in zip(*box)), dtype=fields[f][1].dtype, device="cuda")
            for f, box, _, _ in qs]
    lat, stats = srv.replay(qs, arrivals, outs)
    torch.cuda.synchronize()
    return srv, outs, lat, stats


def _same(a, b):
    return torch.equal(a.contiguous().view(torch.uint8), b.contiguous().view(torch.uint8))


@pytest.mark.parametrize("mode", ["batched_cache", "batched_nocache", "serial"])
def test_results_equal_alone(P, fields, mode):
    qs = _queries(fields, 240, seed=1)
    kw = {"batched_cache": {}, "batched_nocache": {"cache": False}, "serial": {"serial": True, "cache": False}}[mode]
    arrivals = [0.0] * len(qs)  # everything waiting at once: the largest batches
    srv, outs, lat, stats = _run(P, fields, qs, arrivals, **kw)
    assert stats["queries"] == len(qs)
    if mode == "serial":
        assert stats["max_batch"] == 1 and stats["batches"] == len(qs)
    else:
        assert stats["max_batch"] > 1
    for q, o in zip(qs, outs):
        assert _same(o, _alone(P, fields, q)), q
    assert np.all(lat > 0)
    srv.close()


def test_warm_cache_and_poisson_arrivals(P, fields):
    """Replays a stream twice on one server (the second time the caches hold
    partial sums from the first); then a Poisson stream at a high rate."""
    qs = _queries(fields, 200, seed=2, aligned_only=True)
    srv, outs, _, _ = _run(P, fields, qs, [0.0] * len(qs))
    want = [_alone(P, fields, q) for q in qs]
    for o, w in zip(outs, want):
        assert _same(o, w)
    # reversed order: bricks cached at high k serve lower-k queries from scratch
    rq = qs[::-1]
    outs2 = [torch.empty_like(o) for o in outs[::-1]]
    lat, stats = srv.replay(rq, [0.0] * len(rq), outs2)
    torch.cuda.synchronize()
    for o, w in zip(outs2, want[::-1]):
        assert _same(o, w)
    rng = np.random.default_rng(5)
    arr = np.cumsum(rng.exponential(1.0 / 20000.0, len(qs)))
    outs3 = [torch.empty_like(o) for o in outs]
    lat, stats = srv.replay(qs, arr.tolist(), outs3)
    torch.cuda.synchronize()
    for o, w in zip(outs3, want):
        assert _same(o, w)
    assert stats["queries"] == len(qs) and np.all(lat > 0)
    srv.reset_cache()
    srv.close()


def test_matches_oracle(P, fields):
    qs = _queries(fields, 40, seed=3)
    _, outs, _, _ = _run(P, fields, qs, [0.0] * len(qs))
    refs = {}
    for q, o in zip(qs, outs):
        f, (lo, hi), t, k = q
        x, _, tau, _ = fields[f]
        if f not in refs:
            refs[f] = O.Streams(x, tau, nthreads=4)
        kk = k if k else O.query_k(tau, t)
        want = refs[f].retrieve(kk, box=(lo, hi))
        got = o.cpu().numpy()
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), q


def _fixed_bytes(P, fields):
    """Device bytes a server holds before any result (streams, caches, buffers)."""
    budget = 8 << 30
    srv = P.Server(budget)
    for _, _, _, st in fields:
        srv.add_field(st)
    _, stats = srv.replay([(0, ([0, 0, 0], [4, 4, 4]), 0.0, 1)], [0.0])
    srv.close()
    return budget - stats["arena_bytes"]


def test_admission_under_tight_budget(P, fields):
    """A budget that leaves room for about 2.5 of the largest result boxes:
    queries wait for memory, and all complete with the right results."""
    qs = _queries(fields, 120, seed=4)
    biggest = max(int(np.prod([h - l for l, h in zip(*box)])) * fields[f][0].itemsize for f, box, _, _ in qs)
    budget = _fixed_bytes(P, fields) + int(2.5 * biggest) + 4096
    srv, outs, _, stats = _run(P, fields, qs, [0.0] * len(qs), budget=budget)
    assert stats["peak_device_bytes"] <= budget
    assert stats["arena_bytes"] < 3 * biggest
    for q, o in zip(qs, outs):
        assert _same(o, _alone(P, fields, q))
    srv.close()


def test_errors(P, fields):
    srv = P.Server(8 << 30)
    fid = srv.add_field(fields[0][3])
    x, _, tau, st = fields[0]
    full = ([0, 0, 0], list(x.shape))
    with pytest.raises(P.PczError) as e:
        srv.replay([(fid + 5, full, 0.0, 1)], [0.0])
    assert e.value.name == "PC_ERR_ARG"
    with pytest.raises(P.PczError) as e:
        srv.replay([(fid, full, tau[-1] * 0.5, 0)], [0.0])
    assert e.value.name == "PC_ERR_TOL_UNREACHABLE"
    with pytest.raises(P.PczError) as e:
        srv.replay([(fid, full, 0.0, 1), (fid, full, 0.0, 2)], [1.0, 0.5])
    assert e.value.name == "PC_ERR_ARG"
    x2 = S.powerlaw((40, 40), seed=6, dtype=np.float32)
    st2 = P.compress(torch.from_numpy(x2).cuda(), O.tau_decade(O.value_range(x2), 3))
    with pytest.raises(P.PczError) as e:
        srv.add_field(st2)
    assert e.value.name == "PC_ERR_ARG"
    srv.close()
    small = P.Server(_fixed_bytes(P, fields[:1]) + x.nbytes // 2)  # a full box does not fit
    small.add_field(st)
    with pytest.raises(P.PczError) as e:
        small.replay([(0, full, 0.0, 8)], [0.0])
    assert e.value.name == "PC_ERR_OOM"
    small.close()


def test_online_submit_poll_wait(P, fields):
    """Online serving: queries submitted one at a time from one thread while a
    second thread waits for them; every result equals the query run alone, and
    with the cache off (no ordering between batches) batches overlap on the
    device (more than one in flight)."""
    import threading
    import time

    qs = _queries(fields, 300, seed=7)
    want = [_alone(P, fields, q) for q in qs]
    for cache in (False, True):
        srv = P.Server(8 << 30, max_batch=16, cache=cache)
        for _, _, _, st in fields:
            srv.add_field(st)
        outs = [torch.empty_like(w) for w in want]
        tickets = [None] * len(qs)
        lats = [None] * len(qs)
        ready = threading.Semaphore(0)

        def waiter():
            for j in range(len(qs)):
                ready.acquire()
                done, lat = srv.wait(tickets[j], timeout_s=30.0)
                assert done
                lats[j] = lat

        th = threading.Thread(target=waiter)
        th.start()
        rng = np.random.default_rng(8)
        for j, (f, box, t, k) in enumerate(qs):
            tickets[j] = srv.submit(f, box, tau=t, k=k, out=outs[j])
            ready.release()
            if rng.random() < 0.1:
                time.sleep(float(rng.exponential(2e-4)))
        th.join()
        for o, w, q in zip(outs, want, qs):
            assert _same(o, w), q
        assert all(lat is not None and lat > 0 for lat in lats)
        assert srv.poll(tickets[0])[0]
        st = srv.stats()
        assert st["queries"] == len(qs)
        if not cache:
            assert st["max_inflight"] >= 2
        with pytest.raises(P.PczError) as e:
            srv.poll(10 ** 9)
        assert e.value.name == "PC_ERR_ARG"
        srv.close()
