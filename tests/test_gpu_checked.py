"""The bounds-checked build of the search kernel (hnsw_search_params
.check_bounds): on valid graphs it returns what the plain kernel and the
oracle return, bit for bit on integer data, and never raises its violation
flag (stats bit 2).  Its refusals (learned stop, unsupported row sizes) are
host-side errors."""
import numpy as np
import pytest

from paper_1603_09320_gb300 import synth
from _graphs import oracle_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available()
    from paper_1603_09320_gb300 import build, hnsw
    build.build()
    return hnsw


@pytest.mark.parametrize("name,n,storage,k,ef", [("tiny", 10_000, "f32", 10, 32), ("tiny", 10_000, "f32", 100, 256),
                                                 ("sift", 20_000, "bf16", 10, 64), ("sift", 20_000, "f32", 10, 64)])
def test_checked_search_equals_oracle(H, name, n, storage, k, ef):
    import torch
    g, X, blob = oracle_graph(name, n)
    Q = synth.queries(name, 700)
    ix = H.Index(blob, storage)
    q = torch.from_numpy(Q).cuda()
    ids, ds, st = ix.search(q, k, ef, stats=True, check_bounds=True)
    pi, pd = ix.search(q, k, ef)
    torch.cuda.synchronize()
    ids, ds, st = ids.cpu().numpy().view(np.uint32), ds.cpu().numpy(), st.cpu().numpy().view(np.uint32)
    ix.close()
    oi, od, os_ = g.knn_search_batch(Q, k, ef, stats=True)
    np.testing.assert_array_equal(ids, oi)
    np.testing.assert_array_equal(ds.astype(np.float64), od)
    np.testing.assert_array_equal(ids, pi.cpu().numpy().view(np.uint32))
    np.testing.assert_array_equal(st[:, 1], os_[:, 1])
    assert not (st[:, 3] & 4).any()


def test_checked_search_refusals(H):
    import torch
    g, X, blob = oracle_graph("tiny", 10_000)
    ix = H.Index(blob, "fp8")
    q = torch.from_numpy(synth.queries("tiny", 8)).cuda()
    with pytest.raises(H.HnswError) as e:
        ix.search(q, 10, 32, check_bounds=True)  # not built for fp8 rows
    assert e.value.status == 1
    ix.close()
