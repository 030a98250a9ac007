"""The GPU's batched construction and insertion against the oracle's batch
forms (orc_build_batched, orc_insert_batched: Alg. 1 with layer-0
insertions in batches that search the graph as it stood before the batch,
pinned on the CPU to Alg. 1 at batch size one), byte for byte on integer
data, where the kernels' fp32 distances are exact: bulk construction with
Alg. 3, Alg. 4 and Alg. 4 with keepPrunedConnections, and two incremental
insertions into a resident index."""
import numpy as np
import pytest

from paper_1603_09320_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("heuristic,keep", [(True, False), (False, False), (True, True)])
def test_gpu_build_equals_batched_oracle(heuristic, keep):
    import torch
    assert torch.cuda.is_available()
    from oracle import oracle as O
    from paper_1603_09320_gb300 import build, hnsw as H
    build.build()
    p = synth.params("tiny")
    N = 10_000
    X = synth.base("tiny", N)
    u = synth.level_uniforms("tiny", N)
    blob = H.build_graph_gpu(X, u, M=p["M"], Mmax=p["Mmax"], Mmax0=p["Mmax0"], ef_construction=p["efC"],
                             heuristic=heuristic, keep_pruned=keep, n_threads=1)
    ob = O.Graph.build_batched(X, u, n_first=4096, heuristic=heuristic, keep_pruned=keep, **p).to_blob()
    if blob != ob:
        g, o = O.Graph.from_blob(blob), O.Graph.from_blob(ob)
        diff = [i for i in range(N) if g.neighbors(i, 0) != o.neighbors(i, 0)]
        raise AssertionError(f"{len(diff)} layer-0 lists differ, first {diff[:10]}")


def test_gpu_insert_equals_batched_oracle():
    import torch
    assert torch.cuda.is_available()
    from oracle import oracle as O
    from paper_1603_09320_gb300 import build, hnsw as H
    build.build()
    p = synth.params("tiny")
    N, n0 = 10_000, 6000
    X = synth.base("tiny", N)
    u = synth.level_uniforms("tiny", N)
    base = O.Graph.build(X[:n0], u[:n0], **p)
    ix = H.Index(base.to_blob(), "f32")
    ix.reserve(N)
    og = O.Graph.new(X, **p)
    lv = [O.level_from_u(float(x), 1.0 / np.log(p["M"])) for x in u]
    for i in range(n0):
        og.insert(i, lv[i])
    for lo, hi in ((6000, 7000), (7000, N)):
        ix.insert(X[lo:hi], u[lo:hi])
        og.insert_batched(lo, u[lo:hi])
    gb, ob = ix.to_blob(), og.to_blob()
    ix.close()
    if gb != ob:
        g, o = O.Graph.from_blob(gb), O.Graph.from_blob(ob)
        diff = [i for i in range(N) if g.neighbors(i, 0) != o.neighbors(i, 0)]
        raise AssertionError(f"{len(diff)} layer-0 lists differ, first {diff[:10]}")


@pytest.mark.parametrize("keep", [False, True])
def test_gpu_build_shrinks_over_all_of_econn(keep):
    """A batch that sends 301 new links to one list (and to a few filler
    lists): the GPU's reverse-link shrink walks the whole of eConn, as the
    oracle's batch form does (Alg. 1), byte for byte."""
    import torch
    assert torch.cuda.is_available()
    import _hub
    from oracle import oracle as O
    from paper_1603_09320_gb300 import build, hnsw as H
    build.build()
    X, u = _hub.hub_input()
    P = _hub.PARAMS
    blob = H.build_graph_gpu(X, u, M=P["M"], Mmax=P["Mmax"], Mmax0=P["Mmax0"], ef_construction=P["efC"],
                             heuristic=True, keep_pruned=keep, n_threads=1)
    ob = O.Graph.build_batched(X, u, n_first=_hub.N_SEED, keep_pruned=keep, **P).to_blob()
    g = O.Graph.from_blob(blob)
    first, near, far = _hub.ray_ids(X.shape[0])
    if not keep:
        assert g.neighbors(0, 0) == near + [far]
    if blob != ob:
        o = O.Graph.from_blob(ob)
        diff = [i for i in range(X.shape[0]) if g.neighbors(i, 0) != o.neighbors(i, 0)]
        raise AssertionError(f"{len(diff)} layer-0 lists differ, first {diff[:10]}")
