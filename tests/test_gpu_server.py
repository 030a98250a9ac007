"""Continuous-batching server: mixed requests (index, n, k, ef, storage,
rerank) submitted while others run on the GPU return exactly what the same
request returns when searched alone; admission waits for arena memory."""
import threading

import numpy as np
import pytest

from paper_1603_09320_gb300 import synth
from _graphs import oracle_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_1603_09320_gb300 import build, hnsw
    build.build()
    g1, X1, b1 = oracle_graph("tiny", 10_000)
    g2, X2, b2 = oracle_graph("sift", 20_000)
    ixs = [hnsw.Index(b1, "f32"), hnsw.Index(b2, "f32"), hnsw.Index(b2, "bf16", keep_fp32=True)]
    Qs = [synth.queries("tiny", 2000), synth.queries("sift", 2000), synth.queries("sift", 2000)]
    yield hnsw, ixs, Qs
    for ix in ixs:
        ix.close()


def _requests(rng, Qs, n_req):
    reqs = []
    for _ in range(n_req):
        which = int(rng.integers(0, 3))
        n = int(np.exp(rng.uniform(0, np.log(300))))
        s = int(rng.integers(0, Qs[which].shape[0] - n))
        k = int(rng.choice([1, 10, 100]))
        ef = int(rng.integers(k, 257))
        reqs.append((which, Qs[which][s:s + n], k, ef, which == 2))
    return reqs


def _alone(ix, q, k, ef, rerank):
    return ix.search(q, k, ef, rerank=rerank)


@pytest.mark.parametrize("slots,budget", [(8, 0), (3, 1 << 20)])
def test_mixed_requests_equal_alone(setup, slots, budget):
    hnsw, ixs, Qs = setup
    rng = np.random.default_rng(slots)
    reqs = _requests(rng, Qs, 150)
    sv = hnsw.Server(n_slots=slots, memory_budget=budget)
    ids_ = [sv.add_index(ix) for ix in ixs]
    tickets = []

    def submit_half(part):
        for r in part:
            tickets.append((r, sv.submit(ids_[r[0]], r[1], r[2], r[3], rerank=r[4])))

    th = [threading.Thread(target=submit_half, args=(reqs[i::2],)) for i in range(2)]
    for t in th:
        t.start()
    peak_queued = 0
    for t in th:
        t.join()
    peak_queued = max(peak_queued, sv.stats()["queued"])
    lat = []
    for (which, q, k, ef, rr), t in tickets:
        ids, ds, ms = sv.wait(t, timeout_ms=60_000)
        ai, ad = _alone(ixs[which], q, k, ef, rr)
        np.testing.assert_array_equal(ids, ai)
        np.testing.assert_array_equal(ds, ad)
        lat.append(ms)
    st = sv.stats()
    sv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["bytes_in_use"] == 0 and st["in_flight"] == 0 and st["queued"] == 0
    assert max(lat) > 0


def test_request_larger_than_budget_is_rejected(setup):
    hnsw, ixs, Qs = setup
    sv = hnsw.Server(n_slots=2, memory_budget=64 * 1024)
    i = sv.add_index(ixs[1])
    with pytest.raises(hnsw.HnswError) as e:
        sv.submit(i, Qs[1][:1000], 10, 32)  # 512 KB of queries > 64 KB budget
    assert e.value.status == 1
    t = sv.submit(i, Qs[1][:10], 10, 32)
    ids, ds, _ = sv.wait(t, timeout_ms=60_000)
    ai, _ = ixs[1].search(Qs[1][:10], 10, 32)
    np.testing.assert_array_equal(ids, ai)
    sv.close()


def test_replay_equals_alone(setup):
    hnsw, ixs, Qs = setup
    rng = np.random.default_rng(11)
    reqs = _requests(rng, Qs, 60)
    sv = hnsw.Server(n_slots=4)
    ids_ = [sv.add_index(ix) for ix in ixs]
    plan = [(ids_[w], q, k, ef, rr) for (w, q, k, ef, rr) in reqs]
    arrivals = np.cumsum(rng.exponential(1e-4, size=len(plan)))
    res, lat, sub = sv.replay(plan, arrivals)
    sv.close()
    assert (lat > 0).all() and (sub >= arrivals - 1e-6).all()
    for (w, q, k, ef, rr), (ids, ds) in zip(reqs, res):
        ai, ad = ixs[w].search(q, k, ef, rerank=rr)
        np.testing.assert_array_equal(ids, ai)
        np.testing.assert_array_equal(ds, ad)


def test_wait_timeout_and_cancel(setup):
    """Host-side failure paths: a bounded wait on a request still running
    returns HNSW_ETIMEOUT and leaves the request to complete; a request still
    queued behind it is cancelled (its wait returns HNSW_ECANCELED and its
    buffers are not written); an admitted request cannot be cancelled."""
    hnsw, ixs, Qs = setup
    sv = hnsw.Server(n_slots=1)
    a, b = sv.add_index(ixs[1]), sv.add_index(ixs[0])
    big = np.ascontiguousarray(np.tile(Qs[1], (25, 1)))  # 50,000 queries at ef 512: many milliseconds
    ta = sv.submit(a, big, 10, 512)
    tb = sv.submit(b, Qs[0][:100], 10, 32)  # another index: never grouped with ta, queued behind it
    with pytest.raises(hnsw.HnswError) as e:
        sv.wait(ta, timeout_ms=0)
    assert e.value.status == 5  # HNSW_ETIMEOUT; ta is still owned by the server
    sv.cancel(tb)
    with pytest.raises(hnsw.HnswError) as e:
        sv.cancel(ta)  # admitted: on the device
    assert e.value.status == 6
    st = sv.stats()
    assert st["cancelled"] == 1 and st["queued"] == 0
    with pytest.raises(hnsw.HnswError) as e:
        sv.wait(tb)
    assert e.value.status == 7  # HNSW_ECANCELED
    ids, ds, _ = sv.wait(ta)
    ai, ad = _alone(ixs[1], big[:500], 10, 512, False)
    np.testing.assert_array_equal(ids[:500], ai)
    np.testing.assert_array_equal(ds[:500], ad)
    with pytest.raises(hnsw.HnswError) as e:
        sv.cancel(ta)  # consumed
    assert e.value.status == 1
    sv.close()
