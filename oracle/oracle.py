"""ctypes front end of the HNSW oracle (arXiv:1603.09320, Algorithms 1-5).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain single-threaded C restatement
of the paper's algorithms (``hnsw_oracle.c``).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import this
module.  It shares no code with the CUDA library in ``paper_1603_09320_gb300``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
SRC = os.path.join(HERE, "hnsw_oracle.c")
NONE = 0xFFFFFFFF

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "hnsw_oracle.h"))
    ):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
        )
        os.replace(tmp, LIB)
    return LIB


class Stats(C.Structure):
    _fields_ = [("n_dist", C.c_uint64), ("n_hops0", C.c_uint64), ("n_hopsU", C.c_uint64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            vp, u32, u64, i32, f64 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int, C.c_double
            sig = {
                "orc_new": (vp, [vp, u64, u32, i32, u32, u32, u32, u32, f64, i32, i32, i32]),
                "orc_free": (None, [vp]),
                "orc_level_from_u": (i32, [f64, f64]),
                "orc_insert": (i32, [vp, u32, i32]),
                "orc_build": (i32, [vp, vp]),
                "orc_build_batched": (i32, [vp, vp, u64, u32]),
                "orc_build_batched_sizes": (i32, [vp, vp, u64, vp, u64]),
                "orc_insert_batched": (i32, [vp, vp, u64, u64, u32]),
                "orc_knn_search": (i32, [vp, vp, i32, i32, vp, vp, vp]),
                "orc_search_layer": (i32, [vp, vp, vp, i32, i32, i32, vp, vp, vp]),
                "orc_greedy_layer": (u32, [vp, vp, u32, i32, vp]),
                "orc_select_simple": (i32, [vp, vp, vp, i32, i32, vp]),
                "orc_select_heuristic": (i32, [vp, vp, u32, vp, i32, i32, i32, i32, i32, vp]),
                "orc_dist_to": (f64, [vp, vp, u32]),
                "orc_set_data": (i32, [vp, vp]),
                "orc_n": (u64, [vp]),
                "orc_level": (i32, [vp, u32]),
                "orc_enter_point": (u32, [vp]),
                "orc_max_level": (i32, [vp]),
                "orc_neighbors": (i32, [vp, u32, i32, vp, i32]),
                "orc_blob_size": (u64, [vp]),
                "orc_save_blob": (i32, [vp, vp, u64]),
                "orc_load_blob": (vp, [vp, u64, vp]),
                "orc_brute_force": (None, [vp, u64, u32, i32, vp, i32, vp, vp]),
                "orc_knn_search_trace": (i32, [vp, vp, i32, i32, i32, i32, vp, vp, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def level_from_u(u: float, mL: float) -> int:
    return lib().orc_level_from_u(float(u), float(mL))


class Graph:
    """An HNSW multilayer graph held by the oracle."""

    def __init__(self, handle, data: np.ndarray):
        self.h = handle
        self._data = data  # keep the vectors alive for orc_select_* calls on rows

    # ---- construction ----------------------------------------------------
    @classmethod
    def new(cls, data, metric=0, M=8, Mmax=None, Mmax0=None, efC=64, mL=None,
            heuristic=True, extend=False, keep_pruned=False) -> "Graph":
        data = np.ascontiguousarray(data, dtype=np.float32)
        N, d = data.shape
        Mmax = M if Mmax is None else Mmax
        Mmax0 = 2 * M if Mmax0 is None else Mmax0
        mL = 1.0 / np.log(M) if mL is None else mL
        h = lib().orc_new(_p(data), N, d, metric, M, Mmax, Mmax0, efC, float(mL),
                          int(heuristic), int(extend), int(keep_pruned))
        if not h:
            raise ValueError("orc_new rejected the parameters")
        return cls(h, data)

    @classmethod
    def build(cls, data, u, **kw) -> "Graph":
        g = cls.new(data, **kw)
        u = np.ascontiguousarray(u, dtype=np.float64)
        if u.shape[0] != g._data.shape[0]:
            raise ValueError("one u per element")
        if lib().orc_build(g.h, _p(u)) != 0:
            raise RuntimeError("orc_build failed")
        return g

    @classmethod
    def build_batched(cls, data, u, n_first: int = 4096, batch: int = 0, batch_sizes=None, **kw) -> "Graph":
        """Alg. 1 with the layer-0 insertions in batches (orc_build_batched):
        the seed (level >= 1 or id < n_first) first, then the others in
        batches that search the graph as it stood before the batch.  Batch
        sizes: the list `batch_sizes` when given (orc_build_batched_sizes),
        else `batch` elements each, else the growing schedule."""
        g = cls.new(data, **kw)
        u = np.ascontiguousarray(u, dtype=np.float64)
        if u.shape[0] != g._data.shape[0]:
            raise ValueError("one u per element")
        if batch_sizes is not None:
            sz = np.ascontiguousarray(batch_sizes, dtype=np.uint32)
            rc = lib().orc_build_batched_sizes(g.h, _p(u), int(n_first), _p(sz), int(sz.shape[0]))
        else:
            rc = lib().orc_build_batched(g.h, _p(u), int(n_first), int(batch))
        if rc != 0:
            raise RuntimeError("orc_build_batched failed")
        return g

    def insert_batched(self, first: int, u, batch: int = 0) -> None:
        """orc_insert_batched: elements first .. first + len(u) - 1."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        if lib().orc_insert_batched(self.h, _p(u), int(first), int(u.shape[0]), int(batch)) != 0:
            raise RuntimeError("orc_insert_batched failed")

    def insert(self, i: int, level: int) -> None:
        if lib().orc_insert(self.h, i, level) != 0:
            raise RuntimeError("orc_insert failed")

    @classmethod
    def from_blob(cls, blob: bytes) -> "Graph":
        buf = np.frombuffer(blob, dtype=np.uint8)
        err = C.c_int(0)
        h = lib().orc_load_blob(_p(buf), buf.size, C.byref(err))
        if not h:
            raise ValueError(f"orc_load_blob rejected the blob (code {err.value})")
        hdr = np.frombuffer(blob[:128], dtype=np.uint8)
        N = int(hdr[16:24].view(np.uint64)[0])
        d = int(hdr[24:28].view(np.uint32)[0])
        data = np.frombuffer(blob, dtype=np.float32, count=N * d, offset=128).reshape(N, d)
        return cls(h, data)

    def to_blob(self) -> bytes:
        n = lib().orc_blob_size(self.h)
        out = np.zeros(n, dtype=np.uint8)
        r = lib().orc_save_blob(self.h, _p(out), n)
        if r != 0:
            raise RuntimeError(f"orc_save_blob failed ({r})")
        return out.tobytes()

    def with_data(self, data) -> "Graph":
        """A copy of this graph (every link kept) over other N x d vectors."""
        data = np.ascontiguousarray(data, dtype=np.float32)
        if data.shape != self._data.shape:
            raise ValueError("same N x d")
        g = Graph.from_blob(self.to_blob())
        if lib().orc_set_data(g.h, _p(data)) != 0:
            raise RuntimeError("orc_set_data failed")
        g._data = data
        return g

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_free(self.h)
            self.h = None

    # ---- inspection ------------------------------------------------------
    @property
    def N(self) -> int:
        return int(lib().orc_n(self.h))

    @property
    def enter_point(self) -> int:
        return int(lib().orc_enter_point(self.h))

    @property
    def max_level(self) -> int:
        return int(lib().orc_max_level(self.h))

    def level(self, i: int) -> int:
        return int(lib().orc_level(self.h, i))

    def levels(self) -> np.ndarray:
        return np.array([self.level(i) for i in range(self.N)], dtype=np.int64)

    def neighbors(self, i: int, lc: int) -> list:
        out = np.zeros(4096, dtype=np.uint32)
        n = lib().orc_neighbors(self.h, i, lc, _p(out), out.size)
        if n < 0:
            raise ValueError("no such element/layer")
        return out[:n].tolist()

    def dist(self, q, i: int) -> float:
        q = np.ascontiguousarray(q, dtype=np.float32)
        return float(lib().orc_dist_to(self.h, _p(q), i))

    # ---- search ----------------------------------------------------------
    def knn_search(self, q, K: int, ef: int, stats: bool = False):
        """Alg. 5 for one query; returns (ids uint32[K], dists float64[K][, Stats])."""
        q = np.ascontiguousarray(q, dtype=np.float32)
        ids = np.zeros(K, dtype=np.uint32)
        ds = np.zeros(K, dtype=np.float64)
        st = Stats()
        if lib().orc_knn_search(self.h, _p(q), K, ef, _p(ids), _p(ds), C.byref(st)) != 0:
            raise RuntimeError("orc_knn_search failed")
        return (ids, ds, st) if stats else (ids, ds)

    def knn_search_batch(self, Q, K: int, ef: int, stats: bool = False):
        Q = np.ascontiguousarray(Q, dtype=np.float32)
        n = Q.shape[0]
        ids = np.zeros((n, K), dtype=np.uint32)
        ds = np.zeros((n, K), dtype=np.float64)
        sts = np.zeros((n, 3), dtype=np.uint64)
        for i in range(n):
            r = self.knn_search(Q[i], K, ef, stats=True)
            ids[i], ds[i] = r[0], r[1]
            sts[i] = (r[2].n_dist, r[2].n_hops0, r[2].n_hopsU)
        return (ids, ds, sts) if stats else (ids, ds)

    def knn_search_trace(self, q, K: int, ef: int, T: int = 4, max_checks: int = 256):
        """Layer-0 state records (see orc_knn_search_trace): (raw[c][6], topk[c][K])."""
        q = np.ascontiguousarray(q, dtype=np.float32)
        raw = np.zeros((max_checks, 6), dtype=np.float64)
        topk = np.zeros((max_checks, K), dtype=np.uint32)
        nc = C.c_int(0)
        if lib().orc_knn_search_trace(self.h, _p(q), K, ef, T, max_checks, _p(raw), _p(topk), C.byref(nc)) != 0:
            raise RuntimeError("orc_knn_search_trace failed")
        return raw[:nc.value], topk[:nc.value]

    def search_layer(self, q, ep, ef: int, lc: int):
        q = np.ascontiguousarray(q, dtype=np.float32)
        ep = np.ascontiguousarray(np.atleast_1d(ep), dtype=np.uint32)
        cap = max(ef, ep.size) + 2
        ids = np.zeros(cap, dtype=np.uint32)
        ds = np.zeros(cap, dtype=np.float64)
        n = lib().orc_search_layer(self.h, _p(q), _p(ep), ep.size, ef, lc, _p(ids), _p(ds), None)
        return ids[:n], ds[:n]

    def greedy_layer(self, q, ep: int, lc: int) -> int:
        q = np.ascontiguousarray(q, dtype=np.float32)
        return int(lib().orc_greedy_layer(self.h, _p(q), ep, lc, None))

    def select_simple(self, base, cand, M: int):
        base = np.ascontiguousarray(base, dtype=np.float32)
        cand = np.ascontiguousarray(cand, dtype=np.uint32)
        out = np.zeros(max(M, 1), dtype=np.uint32)
        n = lib().orc_select_simple(self.h, _p(base), _p(cand), cand.size, M, _p(out))
        return out[:n].tolist()

    def select_heuristic(self, base, cand, M: int, lc: int = 0, base_id: int = NONE,
                         extend: bool = False, keep_pruned: bool = False):
        base = np.ascontiguousarray(base, dtype=np.float32)
        cand = np.ascontiguousarray(cand, dtype=np.uint32)
        out = np.zeros(max(M, 1), dtype=np.uint32)
        n = lib().orc_select_heuristic(self.h, _p(base), base_id, _p(cand), cand.size, M, lc,
                                       int(extend), int(keep_pruned), _p(out))
        return out[:n].tolist()


def brute_force(data, Q, K: int, metric: int = 0):
    """Exact k-NN by full scan in fp64, key order (distance, id)."""
    data = np.ascontiguousarray(data, dtype=np.float32)
    Q = np.ascontiguousarray(np.atleast_2d(Q), dtype=np.float32)
    N, d = data.shape
    ids = np.zeros((Q.shape[0], K), dtype=np.uint32)
    ds = np.zeros((Q.shape[0], K), dtype=np.float64)
    for i in range(Q.shape[0]):
        lib().orc_brute_force(_p(data), N, d, metric, _p(Q[i]), K,
                              ids[i].ctypes.data_as(C.c_void_p), ds[i].ctypes.data_as(C.c_void_p))
    return ids, ds


def merge_by_key(shard_ids, shard_dists, id_base, K: int):
    """Data-sharded search's merge, by its definition: for each query the K
    smallest keys (distance, global id) of the union of the shards' answers,
    global id = id_base[s] + local id; NONE entries are absent; padded with
    (NONE, +inf).  shard_ids / shard_dists are [S][n][k] arrays."""
    shard_ids = np.asarray(shard_ids, dtype=np.uint64)
    shard_dists = np.asarray(shard_dists, dtype=np.float64)
    S, n, _ = shard_ids.shape
    ids = np.full((n, K), NONE, dtype=np.uint32)
    ds = np.full((n, K), np.inf, dtype=np.float64)
    for q in range(n):
        keys = []
        for s in range(S):
            for j in range(shard_ids.shape[2]):
                if shard_ids[s, q, j] != NONE:
                    keys.append((float(shard_dists[s, q, j]), int(id_base[s]) + int(shard_ids[s, q, j])))
        keys.sort()
        for j, (dd, ii) in enumerate(keys[:K]):
            ids[q, j] = ii
            ds[q, j] = dd
    return ids, ds
