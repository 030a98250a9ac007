"""Data-sharded search on CPU (no GPU): the merge's definition pinned, the
shard ranges, and the exchange step with two gloo ranks.

The merge by key (oracle.merge_by_key) is pinned to exact k-NN: the K
smallest keys of the shards' exact K nearest are the exact K nearest of the
whole data set.  The two-rank test runs the product's all-gather
(sharded.gather_shards) over gloo with each rank's shard answered by the
oracle's Alg. 5 on that shard's own graph (the search itself is the GPU's
and is checked by the -m gpu tests); every rank must end with the oracle's
per-shard searches merged by key."""
import os
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_1603_09320_gb300 import sharded, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_shard_ranges_partition_the_ids():
    for n, w in ((10, 3), (1000, 4), (7, 7), (5, 8)):
        rs = [sharded.shard_range(n, r, w) for r in range(w)]
        assert rs[0][0] == 0 and rs[-1][1] == n
        assert all(rs[i][1] == rs[i + 1][0] for i in range(w - 1))
        assert max(hi - lo for lo, hi in rs) - min(hi - lo for lo, hi in rs) <= 1
    with pytest.raises(ValueError):
        sharded.shard_range(10, 3, 3)


@pytest.mark.parametrize("S", [1, 2, 3, 5])
def test_merge_of_shard_brute_force_is_brute_force(S):
    X = synth.base("tiny", 900)
    Q = synth.queries("tiny", 40)
    k = 10
    bases, si, sd = [], [], []
    for s in range(S):
        lo, hi = sharded.shard_range(900, s, S)
        i, d = O.brute_force(X[lo:hi], Q, k)
        bases.append(lo)
        si.append(i)
        sd.append(d)
    mi, md = O.merge_by_key(np.stack(si), np.stack(sd), bases, k)
    bi, bd = O.brute_force(X, Q, k)
    np.testing.assert_array_equal(mi, bi)
    np.testing.assert_array_equal(md, bd)


def test_merge_pads_when_the_shards_hold_fewer_than_k():
    X = synth.base("tiny", 9)
    Q = synth.queries("tiny", 3)
    a = O.brute_force(X[:4], Q, 6)
    b = O.brute_force(X[4:], Q, 6)
    mi, md = O.merge_by_key(np.stack([a[0], b[0]]), np.stack([a[1], b[1]]), [0, 4], 12)
    bi, bd = O.brute_force(X, Q, 9)
    np.testing.assert_array_equal(mi[:, :9], bi)
    assert (mi[:, 9:] == O.NONE).all() and np.isinf(md[:, 9:]).all()


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from oracle import oracle as O
    from paper_1603_09320_gb300 import sharded, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N, k, ef = 3000, 10, 40
    X = synth.base("tiny", N)
    Q = synth.queries("tiny", 50)
    lo, hi = sharded.shard_range(N, rank, world)
    g = O.Graph.build(X[lo:hi], synth.level_uniforms("tiny", N)[lo:hi], **synth.params("tiny"))
    ids, ds = g.knn_search_batch(Q, k, ef)
    si, sd = sharded.gather_shards(torch.from_numpy(ids.astype(np.int64)), torch.from_numpy(ds))
    bases = [sharded.shard_range(N, r, world)[0] for r in range(world)]
    mi, md = O.merge_by_key(si.numpy(), sd.numpy(), bases, k)
    np.savez(os.path.join(out, f"r{rank}.npz"), ids=mi, ds=md, si=si.numpy())
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_and_merge(tmp_path):
    pytest.importorskip("torch.distributed")
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    r = [np.load(tmp_path / f"r{i}.npz") for i in range(2)]
    N, k, ef = 3000, 10, 40
    X = synth.base("tiny", N)
    Q = synth.queries("tiny", 50)
    u = synth.level_uniforms("tiny", N)
    per = []
    for s in range(2):
        lo, hi = sharded.shard_range(N, s, 2)
        per.append(O.Graph.build(X[lo:hi], u[lo:hi], **synth.params("tiny")).knn_search_batch(Q, k, ef))
    for s in range(2):  # rank order of the gathered answers
        np.testing.assert_array_equal(r[0]["si"][s], per[s][0])
    ei, ed = O.merge_by_key(np.stack([p[0] for p in per]), np.stack([p[1] for p in per]), [0, N // 2], k)
    for x in r:
        np.testing.assert_array_equal(x["ids"], ei)
        np.testing.assert_array_equal(x["ds"], ed)
