"""Two-pass scheduling (descent of all queries, then the layer-0 beams in
order of decreasing descent distance) changes only the order of work: ids,
distances and counters equal the one-pass search and the oracle."""
import numpy as np
import pytest

from paper_1603_09320_gb300 import synth
from _graphs import oracle_graph

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage,keep,rerank", [("f32", False, False), ("bf16", True, True)])
def test_two_pass_equals_one_pass_and_oracle(storage, keep, rerank):
    import torch
    from paper_1603_09320_gb300 import build, hnsw
    build.build()
    g, X, blob = oracle_graph("sift", 20_000)
    ix = hnsw.Index(blob, storage, keep_fp32=keep)
    Q = synth.queries("sift", 20_000)  # above 16,384: two sort chunks
    q = torch.from_numpy(Q).cuda()
    a = ix.search(q, 10, 48, rerank=rerank, stats=True, schedule=1)
    b = ix.search(q, 10, 48, rerank=rerank, stats=True, schedule=2)
    c = ix.search(q, 10, 48, rerank=rerank, stats=True)  # automatic: one pass at this size
    torch.cuda.synchronize()
    for x, y in ((a, b), (a, c)):
        assert torch.equal(x[0], y[0]) and torch.equal(x[1], y[1]) and torch.equal(x[2][:, 1:3], y[2][:, 1:3])
    ids = b[0].cpu().numpy().view(np.uint32)
    ds = b[1].cpu().numpy()
    for i in range(0, 20_000, 997):
        oi, od = g.knn_search(Q[i], 10, 48)
        np.testing.assert_array_equal(ids[i], oi)
        np.testing.assert_array_equal(ds[i].astype(np.float64), od)
    ix.close()
