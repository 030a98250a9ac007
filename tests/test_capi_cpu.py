"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point declared in include/hnsw.h, builds graphs (Alg. 1 + Alg. 4)
and rejects corrupt graph blobs before touching the device."""
import os
import re

import numpy as np
import pytest

from paper_1603_09320_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    from paper_1603_09320_gb300 import build, hnsw
    build.build()
    return hnsw


def test_exports_every_declared_symbol(H):
    hdrs = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]
    names = set()
    for h in hdrs:
        txt = open(h).read()
        names |= set(re.findall(r"^[a-z_ ]*?(?:hnsw_status|void|int|const char\*)\s+\*?(hnsw_\w+)\(", txt, re.M))
    assert names, "no declarations found"
    L = H.lib()
    for n in names:
        assert hasattr(L, n), n
    assert L.hnsw_abi_version() == 2


def test_builder_one_thread_equals_oracle(H, oracle):
    # with one thread the builder is Alg. 1 in id order: byte-identical graph
    for name, n in (("tiny", 3000), ("sift", 2000)):
        p = synth.params(name)
        X = synth.base(name, n)
        u = synth.level_uniforms(name, n)
        g = oracle.Graph.build(X, u, **p)
        b = H.build_graph(X, u, metric=p["metric"], M=p["M"], Mmax=p["Mmax"], Mmax0=p["Mmax0"],
                          ef_construction=p["efC"], n_threads=1)
        assert b == g.to_blob()


def test_builder_simple_selection_equals_oracle(H, oracle):
    p = synth.params("tiny")
    X = synth.base("tiny", 1500)
    u = synth.level_uniforms("tiny", 1500)
    g = oracle.Graph.build(X, u, heuristic=False, **p)
    b = H.build_graph(X, u, M=p["M"], ef_construction=p["efC"], heuristic=False, n_threads=1)
    assert b == g.to_blob()


def test_builder_multithreaded_graph_is_valid(H, oracle):
    # parity unpinned (insertion order is not deterministic): check the
    # invariants via the oracle's validating loader and the recall
    p = synth.params("tiny")
    X = synth.base("tiny", 5000)
    u = synth.level_uniforms("tiny", 5000)
    b = H.build_graph(X, u, M=p["M"], ef_construction=p["efC"], n_threads=4)
    g = oracle.Graph.from_blob(b)
    lv = g.levels()
    assert g.level(g.enter_point) == lv.max()
    for i in range(0, 5000, 37):
        for lc in range(lv[i] + 1):
            nb = g.neighbors(i, lc)
            assert len(nb) <= (16 if lc == 0 else 8)
    Q = synth.queries("tiny", 100)
    bi, _ = oracle.brute_force(X, Q, 10)
    ids, _ = g.knn_search_batch(Q, 10, 128)
    from _graphs import recall
    assert recall(ids, bi) > 0.95


def test_builder_multithreaded_keeps_m_links(H, oracle):
    # Alg. 3 keeps M links whenever it has M candidates, and a shrink keeps
    # Mmax0 >= M: the sequential graph has no element below M links, and the
    # concurrent build (after its sequential start) must not have any either
    p = synth.params("tiny")
    X = synth.base("tiny", 6000)
    u = synth.level_uniforms("tiny", 6000)
    b = H.build_graph(X, u, M=p["M"], ef_construction=p["efC"], heuristic=False, n_threads=8)
    g = oracle.Graph.from_blob(b)
    assert min(len(g.neighbors(i, 0)) for i in range(6000)) >= p["M"]


def test_graph_file_round_trip_and_rejections(H, oracle, tmp_path):
    p = synth.params("tiny")
    X = synth.base("tiny", 2000)
    u = synth.level_uniforms("tiny", 2000)
    b = H.build_graph(X, u, M=p["M"], ef_construction=p["efC"], n_threads=1)
    path = str(tmp_path / "g.hnsw")
    H.save_graph(b, path)
    assert H.load_graph(path) == b
    assert not (tmp_path / "g.hnsw.tmp").exists()
    # the loaded graph is the oracle's own graph (same bytes as its blob)
    assert oracle.Graph.from_blob(H.load_graph(path)).to_blob() == b
    # a flipped payload byte fails the checksum; a truncated file its size
    bad = bytearray(b)
    bad[200] ^= 1
    (tmp_path / "bad.hnsw").write_bytes(bytes(bad))
    with pytest.raises(H.HnswError):
        H.load_graph(str(tmp_path / "bad.hnsw"))
    (tmp_path / "short.hnsw").write_bytes(b[:-16])
    with pytest.raises(H.HnswError):
        H.load_graph(str(tmp_path / "short.hnsw"))
    with pytest.raises(H.HnswError):
        H.load_graph(str(tmp_path / "missing.hnsw"))
    # an invalid blob is not written
    with pytest.raises(H.HnswError):
        H.save_graph(bytes(bad), str(tmp_path / "never.hnsw"))
    assert not (tmp_path / "never.hnsw").exists()


def test_insertion_entry_points_reject_null_arguments_without_gpu(H):
    import ctypes as C
    L = H.lib()
    assert L.hnsw_insert(None, None, 1, None, None) != 0
    assert L.hnsw_reserve(None, 10, None) != 0
    out, n = C.c_void_p(), C.c_uint64()
    assert L.hnsw_index_to_blob(None, C.byref(out), C.byref(n)) != 0
    assert b"null" in H.lib().hnsw_last_error()


def test_gpu_builder_rejects_bad_params_without_gpu(H):
    # parameter checks come before any CUDA call
    X = synth.base("tiny", 10)
    u = np.full(10, 0.5)
    for kw in (dict(M=8, Mmax=4), dict(M=8, ef_construction=2000), dict(M=8, mL=-1.0)):
        with pytest.raises(H.HnswError):
            H.build_graph_gpu(X, u, **kw)
    with pytest.raises(H.HnswError):
        H.build_graph_gpu(np.zeros((10, 300), np.float32), u, M=8)


def test_builder_rejects_bad_params(H):
    X = synth.base("tiny", 10)
    with pytest.raises(H.HnswError):
        H.build_graph(X, np.full(10, 0.5), M=8, Mmax=4)
    with pytest.raises(H.HnswError):
        H.build_graph(X, np.full(10, 0.0), M=8)  # u must be in (0,1]


def test_upload_rejects_corrupt_blob_without_gpu(H, oracle):
    # validation runs on the host before any CUDA call
    g = oracle.Graph.build(synth.base("tiny", 300), synth.level_uniforms("tiny", 300), **synth.params("tiny"))
    b = bytearray(g.to_blob())
    b[300] ^= 0x40
    with pytest.raises(H.HnswError) as e:
        H.Index(bytes(b))
    assert e.value.status == 4
    with pytest.raises(H.HnswError) as e:
        H.Index(bytes(b[:100]))
    assert e.value.status == 4
