"""The multi-rank logic of bench.py on CPU with two gloo ranks: replicas share
one graph (rank 0 builds, the other loads after a barrier), the step time is
the slowest rank's, and the reported rate counts every rank's queries."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, tmp, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import hashlib
    import types

    import torch.distributed as dist

    import bench
    from paper_1603_09320_gb300 import graphs, synth
    graphs.CACHE = tmp  # a private cache directory for this test
    dist.init_process_group("gloo", rank=rank, world_size=world)
    args = types.SimpleNamespace(n_base=300, threads=1)
    X = synth.base("sift", 300)
    u = synth.level_uniforms("sift", 300)
    blob, _ = bench.shared_graph(args, X, u, lambda m: None, rank, dist)
    ms = bench.max_over_ranks(10.0 + rank, dist)
    qps = bench.whole_job_qps(1000, world, ms)
    with open(os.path.join(out, f"r{rank}.txt"), "w") as f:
        f.write(f"{hashlib.sha256(blob).hexdigest()} {ms} {qps}\n")
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    pytest.importorskip("torch.distributed")
    import socket

    import torch.multiprocessing as mp
    from paper_1603_09320_gb300 import build
    build.build()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cache = tmp_path / "cache"
    cache.mkdir()
    mp.start_processes(_rank, args=(2, port, str(cache), str(tmp_path)), nprocs=2, start_method="spawn")
    r0 = open(tmp_path / "r0.txt").read().split()
    r1 = open(tmp_path / "r1.txt").read().split()
    assert r0[0] == r1[0]                      # same graph on both replicas
    assert float(r0[1]) == float(r1[1]) == 11.0  # the slowest rank's time
    assert abs(float(r0[2]) - 2000 / 0.011) < 1e-6 * 2000 / 0.011
