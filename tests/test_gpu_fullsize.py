"""Parity at the full 1M x 128 size, in the launch configuration bench.py
times (10,000 queries per launch), on sampled queries the oracle answers one
by one on the same graph.  Integer coordinates: ids and distances must be
identical."""
import numpy as np
import pytest

from paper_1603_09320_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage,keep,rerank,ef", [("f32", False, False, 64), ("bf16", True, True, 64),
                                                    ("f32", False, False, 400)])
def test_sift_1m_sampled(storage, keep, rerank, ef):
    import torch
    from oracle import oracle as O
    from paper_1603_09320_gb300 import build, graphs, hnsw
    build.build()
    N = 1_000_000
    blob, _ = graphs.build_or_load("sift", N)
    Q = synth.queries("sift", 10_000)
    ix = hnsw.Index(blob, storage, keep_fp32=keep)
    q = torch.from_numpy(Q).cuda()
    ids, ds, st = ix.search(q, 10, ef, rerank=rerank, stats=True)
    torch.cuda.synchronize()
    ids = ids.cpu().numpy().view(np.uint32)
    ds = ds.cpu().numpy()
    st = st.cpu().numpy().view(np.uint32)
    ix.close()
    g = _oracle_graph(blob)
    rng = np.random.default_rng(0)
    sample = np.concatenate([[0, 9999], rng.choice(10_000, size=38, replace=False)])
    for i in sample:
        oi, od, ost = g.knn_search(Q[i], 10, ef, stats=True)
        np.testing.assert_array_equal(ids[i], oi)
        np.testing.assert_array_equal(ds[i].astype(np.float64), od)
        assert st[i, 1] == ost.n_hops0 and st[i, 2] == ost.n_hopsU


_cache = {}


def _oracle_graph(blob):
    from oracle import oracle as O
    key = id(blob)
    if key not in _cache:
        _cache.clear()
        _cache[key] = O.Graph.from_blob(blob)
    return _cache[key]
