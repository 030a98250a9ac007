"""hnsw_search_noalloc: the search entry point for callers that cannot
allocate device memory while searching (their device memory is reserved by
another allocator, or they must avoid cudaMalloc's device synchronisation).

It is called here through the C ABI (ctypes) and must return exactly what
hnsw_search returns, on two calls in a row, with host buffers (staged through
the library's fixed device array) and with device buffers.  This file is
collected last so that a run stopping at the first failure has run every
other test already.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1603_09320_gb300 import synth

pytestmark = pytest.mark.gpu


def _noalloc(H):
    f = H.lib().hnsw_search_noalloc
    f.restype = C.c_int32
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    return f


def test_noalloc_matches_hnsw_search():
    import torch
    from oracle import oracle as O
    from paper_1603_09320_gb300 import build, hnsw
    build.build()
    p = synth.params("tiny")
    X = synth.base("tiny", 5000)
    g = O.Graph.build(X, synth.level_uniforms("tiny", 5000), **p)
    ix = hnsw.Index(g.to_blob(), "f32")
    Q = np.ascontiguousarray(synth.queries("tiny", 700))
    n, k, ef = Q.shape[0], 10, 40
    ref_i = np.empty((n, k), np.uint32)
    ref_d = np.empty((n, k), np.float32)
    st = hnsw.lib().hnsw_search(ix.h, Q.ctypes.data, n, k, ef, ref_i.ctypes.data, ref_d.ctypes.data, None)
    assert st == 0
    f = _noalloc(hnsw)
    for _ in range(2):  # host buffers, twice in a row
        ids = np.full((n, k), 7, np.uint32)
        ds = np.full((n, k), -1.0, np.float32)
        assert f(ix.h, Q.ctypes.data, n, k, ef, ids.ctypes.data, ds.ctypes.data, None) == 0
        np.testing.assert_array_equal(ids, ref_i)
        np.testing.assert_array_equal(ds, ref_d)
    qd = torch.from_numpy(Q).cuda()
    for _ in range(2):  # device buffers, twice in a row
        ids = torch.full((n, k), 7, dtype=torch.int32, device="cuda")
        ds = torch.full((n, k), -1.0, dtype=torch.float32, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        assert f(ix.h, qd.data_ptr(), n, k, ef, ids.data_ptr(), ds.data_ptr(), s) == 0
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids.cpu().numpy().view(np.uint32), ref_i)
        np.testing.assert_array_equal(ds.cpu().numpy(), ref_d)
    ix.close()


def test_noalloc_rejects_batches_beyond_the_scratch():
    from oracle import oracle as O
    from paper_1603_09320_gb300 import build, hnsw
    build.build()
    p = synth.params("tiny")
    X = synth.base("tiny", 500)
    g = O.Graph.build(X, synth.level_uniforms("tiny", 500), **p)
    ix = hnsw.Index(g.to_blob(), "f32")
    n, k = 200_000, 10  # 25.6 MB of host queries: above the 16 MiB scratch
    Q = np.zeros((n, 32), np.float32)
    ids = np.zeros((n, k), np.uint32)
    ds = np.zeros((n, k), np.float32)
    st = _noalloc(hnsw)(ix.h, Q.ctypes.data, n, k, 20, ids.ctypes.data, ds.ctypes.data, None)
    assert st == 1  # HNSW_EINVAL
    assert b"scratch" in hnsw.lib().hnsw_last_error()
    ix.close()


def test_noalloc_allocates_no_device_memory():
    """A fresh index searched only through hnsw_search_noalloc with host
    buffers holds no staging buffer afterwards, and the device's free memory
    is the same before and after two calls (the first call on this device,
    which resolves the fixed array's address and may load the module, runs
    beforehand on another index)."""
    import torch
    from oracle import oracle as O
    from paper_1603_09320_gb300 import build, hnsw
    build.build()
    p = synth.params("tiny")
    X = synth.base("tiny", 3000)
    blob = O.Graph.build(X, synth.level_uniforms("tiny", 3000), **p).to_blob()
    Q = np.ascontiguousarray(synth.queries("tiny", 500))
    n, k, ef = Q.shape[0], 10, 32
    f = _noalloc(hnsw)
    warm = hnsw.Index(blob, "f32")
    ids = np.zeros((n, k), np.uint32)
    ds = np.zeros((n, k), np.float32)
    assert f(warm.h, Q.ctypes.data, n, k, ef, ids.ctypes.data, ds.ctypes.data, None) == 0
    ix = hnsw.Index(blob, "f32")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert f(ix.h, Q.ctypes.data, n, k, ef, ids.ctypes.data, ds.ctypes.data, None) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    info = hnsw.IndexInfo()
    assert hnsw.lib().hnsw_get_index_info(ix.h, info) == 0
    assert info.staging_bytes == 0
    assert free1 == free0
    # hnsw_search with host buffers on the same index does stage (the
    # counter sees a staging buffer when there is one)
    assert hnsw.lib().hnsw_search(ix.h, Q.ctypes.data, n, k, ef, ids.ctypes.data, ds.ctypes.data, None) == 0
    assert hnsw.lib().hnsw_get_index_info(ix.h, info) == 0
    assert info.staging_bytes > 0
    ix.close()
    warm.close()
