"""Data-sharded search over several ranks (Section 6 discusses distributing
HNSW by partitioning the data; it notes that partitioning scales throughput
less well than replicas, which is why replicas are the default multi-GPU
form).

Rank r of S holds the graph of one contiguous shard of the data, global ids
[base_r, base_r + N_r), built over that shard alone.  A query batch is
searched by every rank on its own graph; the ranks' k nearest (local ids and
distances, [n][k] each) are gathered into [S][n][k] on every rank (the one
exchange of the path: an all-gather over the process group), and the k
smallest keys (distance, global id) of the union are kept by the merge
kernel (hnsw_merge_topk).  Every step runs in the library's kernels; this
module only arranges shards, gathers and calls.
"""
from __future__ import annotations

import numpy as np

from . import hnsw


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Global ids [lo, hi) of shard `rank` of `world` contiguous shards of n
    elements (sizes differ by at most one)."""
    if not (0 <= rank < world):
        raise ValueError("rank outside [0, world)")
    return n * rank // world, n * (rank + 1) // world


def gather_shards(ids, dists, group=None):
    """All-gathers this rank's [n][k] results into [S][n][k] tensors, rank
    order (every rank must pass the same n and k)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    gi = [torch.empty_like(ids) for _ in range(world)]
    gd = [torch.empty_like(dists) for _ in range(world)]
    dist.all_gather(gi, ids.contiguous(), group=group)
    dist.all_gather(gd, dists.contiguous(), group=group)
    return torch.stack(gi), torch.stack(gd)


class ShardedIndex:
    """This rank's shard of a data-sharded index on the current CUDA device."""

    def __init__(self, shard_blob: bytes, id_base: int, n_total: int, group=None, storage: str = "f32",
                 keep_fp32: bool = False):
        import torch.distributed as dist
        self.index = hnsw.Index(shard_blob, storage, keep_fp32=keep_fp32)
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        lo, hi = shard_range(n_total, self.rank, self.world)
        if id_base != lo or self.index.info.N != hi - lo:
            raise ValueError("the shard's graph does not hold this rank's contiguous range")
        self.bases = np.array([shard_range(n_total, r, self.world)[0] for r in range(self.world)], np.uint32)

    def search(self, queries, k: int, ef: int, rerank: bool = False):
        """Every rank passes the same queries (CUDA tensor [n][d]); every rank
        returns the global k nearest: (ids as int32 viewed uint32, dists)."""
        ids, ds = self.index.search(queries, k, ef, rerank=rerank)
        si, sd = gather_shards(ids, ds, self.group)
        return hnsw.merge_topk(si, sd, self.bases, k)

    def close(self) -> None:
        self.index.close()
