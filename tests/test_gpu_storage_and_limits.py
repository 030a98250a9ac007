"""GPU parity of the quantised storage forms and of the kernel's size
limits against the oracle (same graph; kept in a file collected after the
other search tests).

* Without rerank a quantised index returns the distances to its decoded rows
  (oracle/quant_oracle.py: round-to-nearest-even codes, fp8-e4m3 with the
  row scale max|x| / 448): relative error <= 1e-5 for every returned id (for
  cosine with the floor 0.12 of the fp32 bound), and the oracle's search of
  the same graph over those rows agrees (overlap >= 0.999).
* At k = 1024 and ef' = 1024 (the kernel's limits) ids, distances and
  layer-0 expansion counts are bit-exact on integer data.
"""
import numpy as np
import pytest

from paper_1603_09320_gb300 import synth
from _graphs import oracle_graph
from test_gpu_search import COSINE_FLOOR, _tolerance_check, gpu_search, oracle_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available()
    from paper_1603_09320_gb300 import build, hnsw
    build.build()
    return hnsw


@pytest.mark.parametrize("k,ef", [(1024, 1024), (10, 1024), (1024, 1)])
def test_tiny_bit_exact_at_the_limits(H, k, ef):
    # the largest k and ef' = max(ef, k) the kernel takes (1024): W, the
    # visited set (which overflows here) and the output at their maximum
    g, X, blob = oracle_graph("tiny", 10_000)
    Q = synth.queries("tiny", 200)
    gi, gd, gs = gpu_search(H, blob, Q, k, ef, stats=True)
    oi, od, os_ = oracle_batch(g, Q, k, ef)
    np.testing.assert_array_equal(gi, oi)
    np.testing.assert_array_equal(gd.astype(np.float64), od)
    np.testing.assert_array_equal(gs[:, 1], os_[:, 1])


@pytest.mark.parametrize("storage,name", [("fp8", "sift"), ("fp8", "glove"), ("bf16", "lowd"), ("f16", "lowd"),
                                          ("bf16", "glove")])
def test_quantised_distances_are_those_of_the_decoded_rows(H, storage, name):
    # without rerank a quantised index returns distances to its decoded rows
    # (round-to-nearest-even codes; fp8 with the row scale max|x| / 448): the
    # oracle searches the same graph over the rows its own quantiser decodes
    from oracle import quant_oracle as QO
    g, X, blob = oracle_graph(name, 8000 if name == "glove" else 20_000)
    h = g.with_data(QO.decoded_rows(storage, X))
    Q = synth.queries(name, 300)
    gi, gd = gpu_search(H, blob, Q, 10, 96, storage=storage)
    oi, od, _ = oracle_batch(h, Q, 10, 96)
    ex = np.array([[h.dist(Q[i], int(j)) for j in gi[i]] for i in range(len(Q))])
    floor = COSINE_FLOOR if name == "glove" else 0.0
    err = np.abs(gd.astype(np.float64) - ex) / np.maximum(np.abs(ex), max(floor, 1e-30))
    assert err.max() <= 1e-5, err.max()
    _tolerance_check(gi, gd, oi, od, d_floor=floor)
