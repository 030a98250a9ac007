"""Incremental insertion into a resident index (hnsw_reserve / hnsw_insert /
hnsw_index_to_blob).

Pinned against the oracle:
* an uploaded graph read back with hnsw_index_to_blob is the oracle's blob,
  byte for byte;
* the upper layers after insertion equal the oracle's sequential Alg. 1 over
  all elements, list by list: layers >= 1 only involve elements of level
  >= 1 in id order, which the insertion processes one at a time exactly as
  Alg. 1 does (integer-valued data: fp32 distances are exact);
* layer 0 (batch insertion) passes the validating loader, keeps the caps,
  and reaches the oracle graph's reachability and recall within a small
  margin; its byte-for-byte parity with the oracle's batch form is checked in
  test_gpu_build_exact.py.
Concurrent searches during insertion return valid results, and afterwards
the live index searches exactly like a fresh upload of its own blob.
"""
import threading

import numpy as np
import pytest

from paper_1603_09320_gb300 import synth
from _graphs import recall

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available()
    from paper_1603_09320_gb300 import build, hnsw
    build.build()
    return hnsw


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    return oracle


def tiny(n):
    p = synth.params("tiny")
    return p, synth.base("tiny", n), synth.level_uniforms("tiny", n)


def reachable(g):
    seen = np.zeros(g.N, dtype=bool)
    stack = [g.enter_point]
    seen[g.enter_point] = True
    while stack:
        i = stack.pop()
        for j in g.neighbors(i, 0):
            if not seen[j]:
                seen[j] = True
                stack.append(j)
    return int(seen.sum())


def search(H, ix, Q, k, ef):
    import torch
    ids, ds = ix.search(torch.from_numpy(Q).cuda(), k, ef)
    torch.cuda.synchronize()
    return ids.cpu().numpy().view(np.uint32), ds.cpu().numpy()


@pytest.mark.parametrize("storage,keep", [("f32", False), ("bf16", True)])
def test_index_to_blob_is_the_uploaded_graph(H, O, storage, keep):
    p, X, u = tiny(5000)
    g = O.Graph.build(X, u, **p)
    blob = g.to_blob()
    ix = H.Index(blob, storage, keep_fp32=keep)
    assert ix.to_blob() == blob
    ix.reserve(8000)  # reallocation keeps the graph
    assert ix.to_blob() == blob
    ix.close()


def test_insert_upper_layers_equal_sequential_alg1(H, O):
    p, X, u = tiny(10_000)
    n0 = 6000
    base = O.Graph.build(X[:n0], u[:n0], **p)
    full = O.Graph.build(X, u, **p)  # sequential Alg. 1 over all elements
    ix = H.Index(base.to_blob(), "f32")
    ix.reserve(10_000)
    for lo, hi in ((6000, 7000), (7000, 10_000)):
        assert list(ix.insert(X[lo:hi], u[lo:hi])) == list(range(lo, hi))
    g = O.Graph.from_blob(ix.to_blob())  # validating loader
    assert g.enter_point == full.enter_point and g.max_level == full.max_level
    lv = g.levels()
    assert np.array_equal(lv, full.levels())
    for i in np.nonzero(lv > 0)[0]:
        for lc in range(1, int(lv[i]) + 1):
            assert g.neighbors(int(i), lc) == full.neighbors(int(i), lc), (i, lc)
    for i in range(10_000):
        nb = g.neighbors(i, 0)
        assert 1 <= len(nb) <= p["Mmax0"] and i not in nb and len(set(nb)) == len(nb)
    assert reachable(g) >= reachable(full) - 20
    Q = synth.queries("tiny", 500)
    gt, _ = O.brute_force(X, Q, 10)
    fi = H.Index(full.to_blob(), "f32")
    for ef in (16, 32, 64):
        assert recall(search(H, ix, Q, 10, ef)[0], gt) >= recall(search(H, fi, Q, 10, ef)[0], gt) - 0.02
    fi.close()
    ix.close()


def test_insert_into_bf16_index_with_rerank(H, O):
    # construction reads the fp32 copy, so the graph is the one an fp32
    # index gets; bf16 holds these integers exactly, so the searches agree too
    p, X, u = tiny(8000)
    base = O.Graph.build(X[:5000], u[:5000], **p).to_blob()
    ib = H.Index(base, "bf16", keep_fp32=True)
    i32 = H.Index(base, "f32")
    for ix in (ib, i32):
        ix.reserve(8000)
        ix.insert(X[5000:6500], u[5000:6500])
        ix.insert(X[6500:], u[6500:])
        assert ix.info.N == 8000
    assert ib.to_blob() == i32.to_blob()
    Q = synth.queries("tiny", 300)
    import torch
    q = torch.from_numpy(Q).cuda()
    ids_b, ds_b = ib.search(q, 10, 64, rerank=True)
    ids_f, ds_f = i32.search(q, 10, 64)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ids_b.cpu().numpy(), ids_f.cpu().numpy())
    np.testing.assert_array_equal(ds_b.cpu().numpy(), ds_f.cpu().numpy())
    ib.close()
    i32.close()


def test_searches_during_insertion_and_snapshot_equivalence(H, O):
    import torch
    p, X, u = tiny(10_000)
    base = O.Graph.build(X[:4000], u[:4000], **p)
    ix = H.Index(base.to_blob(), "f32")
    ix.reserve(10_000)
    Q = synth.queries("tiny", 256)
    dev = torch.cuda.current_device()
    errors, seen_n = [], []
    done = threading.Event()

    def reader():
        try:
            torch.cuda.set_device(dev)
            s = torch.cuda.Stream()
            q = torch.from_numpy(Q).cuda()
            while not done.is_set():
                n_before = int(ix.info.N)
                ids, ds = ix.search(q, 10, 32, stream=s)
                s.synchronize()
                a = ids.cpu().numpy().view(np.uint32)
                d = ds.cpu().numpy()
                assert (a < 10_000).all()
                assert (np.diff(d, axis=1) >= 0).all()
                assert all(len(set(r.tolist())) == 10 for r in a)
                seen_n.append((n_before, int(a.max())))
        except Exception as e:  # reported on the main thread
            errors.append(e)

    th = threading.Thread(target=reader)
    th.start()
    try:
        for lo in range(4000, 10_000, 1500):
            ix.insert(X[lo:lo + 1500], u[lo:lo + 1500])
    finally:
        done.set()
        th.join()
    assert not errors, errors[0]
    assert len(seen_n) > 0
    # the live index searches exactly like a fresh upload of its own graph
    fresh = H.Index(ix.to_blob(), "f32")
    a1, d1 = search(H, ix, Q, 10, 48)
    a2, d2 = search(H, fresh, Q, 10, 48)
    np.testing.assert_array_equal(a1, a2)
    np.testing.assert_array_equal(d1, d2)
    # as good as the oracle's sequential graph over all elements
    gt, _ = O.brute_force(X, Q, 10)
    full = O.Graph.build(X, u, **p)
    ids_o, _ = full.knn_search_batch(Q, 10, 48)
    assert recall(a1, gt) >= recall(ids_o, gt) - 0.02
    fresh.close()
    ix.close()


def test_insert_cosine(H, O):
    # unit-normalised data, cosine distance: a valid graph as good as the
    # oracle's sequential one over all elements
    p = dict(synth.params("glove"))
    p["efC"] = 100
    N, n0 = 6000, 4000
    X = synth.base("glove", N)
    u = synth.level_uniforms("glove", N)
    base = O.Graph.build(X[:n0], u[:n0], **p)
    full = O.Graph.build(X, u, **p)
    ix = H.Index(base.to_blob(), "f32")
    ix.reserve(N)
    ix.insert(X[n0:], u[n0:])
    g = O.Graph.from_blob(ix.to_blob())
    lv = g.levels()
    for i in np.nonzero(lv > 0)[0]:  # upper layers: sequential Alg. 1 (fp32 vs fp64 ties aside)
        assert len(g.neighbors(int(i), 1)) <= p["Mmax"]
    assert reachable(g) >= reachable(full) - 0.002 * N
    Q = synth.queries("glove", 300)
    gt, _ = O.brute_force(X, Q, 10, metric=1)
    fi = H.Index(full.to_blob(), "f32")
    for ef in (32, 64):
        assert recall(search(H, ix, Q, 10, ef)[0], gt) >= recall(search(H, fi, Q, 10, ef)[0], gt) - 0.02
    fi.close()
    ix.close()


def test_insert_rejections(H, O):
    p, X, u = tiny(3000)
    base = O.Graph.build(X[:2000], u[:2000], **p)
    ix = H.Index(base.to_blob(), "f32")
    with pytest.raises(H.HnswError):  # no capacity reserved
        ix.insert(X[2000:2100], u[2000:2100])
    ix.reserve(2500)
    with pytest.raises(H.HnswError):  # beyond the capacity
        ix.insert(X[2000:], u[2000:])
    with pytest.raises(H.HnswError):  # level draw outside (0, 1]
        ix.insert(X[2000:2010], np.zeros(10))
    assert ix.info.N == 2000
    ix.insert(X[2000:2500], u[2000:2500])
    assert ix.info.N == 2500
    ix.close()
    qb = H.Index(base.to_blob(), "bf16")  # no fp32 copy
    qb.reserve(2500)
    with pytest.raises(H.HnswError):
        qb.insert(X[2000:2100], u[2000:2100])
    qb.close()
