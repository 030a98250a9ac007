"""Data-sharded search on the GPU: each shard's graph searched by the search
kernel, the per-shard answers merged by hnsw_merge_topk, against the
oracle's Alg. 5 on each shard's graph merged by key (oracle.merge_by_key,
pinned on CPU to exact k-NN).  Integer coordinates: bit-exact ids and
distances."""
import ctypes as C

import numpy as np
import pytest

from paper_1603_09320_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available()
    from paper_1603_09320_gb300 import build, hnsw
    build.build()
    return hnsw


def _shards(name, N, S):
    from oracle import oracle as O
    from paper_1603_09320_gb300 import sharded
    X = synth.base(name, N)
    u = synth.level_uniforms(name, N)
    out = []
    for s in range(S):
        lo, hi = sharded.shard_range(N, s, S)
        out.append((lo, O.Graph.build(X[lo:hi], u[lo:hi], **synth.params(name))))
    return out


@pytest.mark.parametrize("name,N,S,k,ef,storage", [("sift", 20_000, 2, 10, 64, "f32"),
                                                   ("sift", 20_000, 3, 10, 48, "bf16"),
                                                   ("tiny", 10_000, 5, 100, 128, "f32"),
                                                   ("tiny", 12, 2, 16, 16, "f32")])
def test_shards_merged_equal_the_oracle(H, name, N, S, k, ef, storage):
    import torch
    from oracle import oracle as O
    shards = _shards(name, N, S)
    Q = synth.queries(name, 777)
    q = torch.from_numpy(Q).cuda()
    gi, gd = [], []
    for lo, g in shards:
        ix = H.Index(g.to_blob(), storage)
        ids, ds = ix.search(q, k, ef)
        gi.append(ids)
        gd.append(ds)
        torch.cuda.synchronize()
        ix.close()
    bases = [lo for lo, _ in shards]
    mi, md = H.merge_topk(torch.stack(gi), torch.stack(gd), bases, k)
    torch.cuda.synchronize()
    per = [g.knn_search_batch(Q, k, ef) for _, g in shards]
    ei, ed = O.merge_by_key(np.stack([p[0] for p in per]), np.stack([p[1] for p in per]), bases, k)
    np.testing.assert_array_equal(mi.cpu().numpy().view(np.uint32), ei)
    np.testing.assert_array_equal(md.cpu().numpy().astype(np.float64), ed)


def test_merge_rejects_bad_arguments(H):
    import torch
    ids = torch.zeros((2, 4, 3), dtype=torch.int32, device="cuda")
    ds = torch.zeros((2, 4, 3), dtype=torch.float32, device="cuda")
    L = H.lib()
    out_i = torch.empty((4, 3), dtype=torch.int32, device="cuda")
    out_d = torch.empty((4, 3), dtype=torch.float32, device="cuda")
    base = np.zeros(40, np.uint32)
    for S, k in ((0, 3), (33, 3), (2, 0), (2, 1025)):
        assert L.hnsw_merge_topk(ids.data_ptr(), ds.data_ptr(), S, base.ctypes.data, 4, k, out_i.data_ptr(),
                                 out_d.data_ptr(), None) == 1
    host = np.zeros((4, 3), np.uint32)
    assert L.hnsw_merge_topk(ids.data_ptr(), ds.data_ptr(), 2, base.ctypes.data, 4, 3, host.ctypes.data,
                             out_d.data_ptr(), None) == 1
    assert b"device memory" in L.hnsw_last_error()


def test_sharded_index_one_rank_over_nccl(H):
    # the whole path of ShardedIndex (local search, all-gather, merge) with a
    # single rank: the answer is the shard's own, ids offset by its base (0)
    import socket

    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_1603_09320_gb300 import sharded
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        (lo, g), = _shards("sift", 5000, 1)
        si = sharded.ShardedIndex(g.to_blob(), lo, 5000)
        Q = synth.queries("sift", 300)
        ids, ds = si.search(torch.from_numpy(Q).cuda(), 10, 32)
        torch.cuda.synchronize()
        si.close()
        oi, od = g.knn_search_batch(Q, 10, 32)
        np.testing.assert_array_equal(ids.cpu().numpy().view(np.uint32), oi)
        np.testing.assert_array_equal(ds.cpu().numpy().astype(np.float64), od)
    finally:
        dist.destroy_process_group()
