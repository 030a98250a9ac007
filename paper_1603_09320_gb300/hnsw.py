"""Thin Python binding of the C ABI in include/hnsw.h (argument marshalling only).

Every step of the search runs in the CUDA kernels of libhnsw_gb300.so; this
module only converts arguments.  Loading fails loudly when the library has not
been built (``python -m paper_1603_09320_gb300.build``): there is no fallback.
Buffers may be numpy arrays (host) or torch tensors (host or CUDA).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

NO_ID = 0xFFFFFFFF
L2SQ, COSINE = 0, 1
F32, BF16, FP8E4M3, F16 = 0, 1, 2, 3
DTYPES = {"f32": F32, "bf16": BF16, "fp8": FP8E4M3, "f16": F16}

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ECORRUPT", 5: "ETIMEOUT", 6: "EBUSY", 7: "ECANCELED"}


class HnswError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class BuildParams(C.Structure):
    _fields_ = [("M", C.c_uint32), ("Mmax", C.c_uint32), ("Mmax0", C.c_uint32),
                ("ef_construction", C.c_uint32), ("mL", C.c_double), ("heuristic", C.c_int32),
                ("extend_candidates", C.c_int32), ("keep_pruned", C.c_int32), ("n_threads", C.c_int32)]


class IndexInfo(C.Structure):
    _fields_ = [("N", C.c_uint64), ("d", C.c_uint32), ("d_pad", C.c_uint32), ("row_bytes", C.c_uint32),
                ("metric", C.c_int32), ("storage", C.c_int32), ("has_fp32", C.c_int32),
                ("M", C.c_uint32), ("Mmax", C.c_uint32), ("Mmax0", C.c_uint32), ("max_level", C.c_int32),
                ("enter_point", C.c_uint32), ("n_upper_rows", C.c_uint64), ("device_bytes", C.c_uint64),
                ("staging_bytes", C.c_uint64)]


class SearchParams(C.Structure):
    _fields_ = [("k", C.c_int32), ("ef", C.c_int32), ("rerank", C.c_int32), ("visited_log2", C.c_int32),
                ("stop_threshold", C.c_float), ("stop_period", C.c_int32), ("schedule", C.c_int32),
                ("check_bounds", C.c_int32)]


class StopTrainParams(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("weight_decay", C.c_float), ("seed", C.c_uint64)]


class ServerParams(C.Structure):
    _fields_ = [("n_slots", C.c_int32), ("memory_budget", C.c_uint64)]


class Request(C.Structure):
    _fields_ = [("index", C.c_int32), ("n", C.c_int64), ("k", C.c_int32), ("ef", C.c_int32), ("rerank", C.c_int32),
                ("stop_threshold", C.c_float), ("stop_period", C.c_int32), ("queries", C.c_void_p),
                ("out_ids", C.c_void_p), ("out_dists", C.c_void_p)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("queued", C.c_uint64), ("in_flight", C.c_uint64), ("bytes_in_use", C.c_uint64),
                ("budget", C.c_uint64), ("cancelled", C.c_uint64)]


class QueryStats(C.Structure):
    _fields_ = [("n_eval", C.c_uint32), ("n_exp0", C.c_uint32), ("n_stepU", C.c_uint32), ("flags", C.c_uint32)]


_lib = None
STOP_NPARAM = 4673


def lib_path() -> str:
    return _build.LIB


def lib():
    """Loads libhnsw_gb300.so (raises if it is missing)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: run python -m paper_1603_09320_gb300.build")
        L = C.CDLL(path)
        vp, u32, u64, i32, i64 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int32, C.c_int64
        sig = {
            "hnsw_build": (i32, [vp, u64, u32, i32, C.POINTER(BuildParams), vp, C.POINTER(vp), C.POINTER(u64)]),
            "hnsw_free_blob": (None, [vp]),
            "hnsw_save_blob": (i32, [vp, u64, C.c_char_p]),
            "hnsw_reserve": (i32, [vp, u64, vp]),
            "hnsw_insert": (i32, [vp, vp, u64, vp, vp]),
            "hnsw_index_to_blob": (i32, [vp, C.POINTER(vp), C.POINTER(u64)]),
            "hnsw_load_blob": (i32, [C.c_char_p, C.POINTER(vp), C.POINTER(u64)]),
            "hnsw_build_gpu": (i32, [vp, u64, u32, i32, C.POINTER(BuildParams), vp, vp, C.POINTER(vp),
                                     C.POINTER(u64)]),
            "hnsw_upload_index": (i32, [vp, u64, i32, i32, vp, C.POINTER(vp)]),
            "hnsw_free_index": (i32, [vp]),
            "hnsw_get_index_info": (i32, [vp, C.POINTER(IndexInfo)]),
            "hnsw_search": (i32, [vp, vp, i64, i32, i32, vp, vp, vp]),
            "hnsw_search_ex": (i32, [vp, C.POINTER(SearchParams), vp, i64, vp, vp, vp, vp]),
            "hnsw_debug_hold_decisions": (i32, [vp, i32]),
            "hnsw_last_error": (C.c_char_p, []),
            "hnsw_set_stop_model": (i32, [vp, vp, vp]),
            "hnsw_clear_stop_model": (i32, [vp]),
            "hnsw_search_trace": (i32, [vp, C.POINTER(SearchParams), vp, i64, i32, vp, vp, vp, vp, vp, vp, vp, vp]),
            "hnsw_stop_grad": (i32, [vp, vp, i64, vp, vp, vp, vp, vp]),
            "hnsw_stop_train": (i32, [vp, vp, i64, C.POINTER(StopTrainParams), vp, vp, vp, vp, vp]),
            "hnsw_abi_version": (i32, []),
            "hnsw_merge_topk": (i32, [vp, vp, i32, vp, i64, i32, vp, vp, vp]),
            "hnsw_server_create": (i32, [C.POINTER(ServerParams), C.POINTER(vp)]),
            "hnsw_server_add_index": (i32, [vp, vp, C.POINTER(i32)]),
            "hnsw_server_submit": (i32, [vp, C.POINTER(Request), C.POINTER(u64)]),
            "hnsw_server_poll": (i32, [vp, u64, C.POINTER(i32)]),
            "hnsw_server_wait": (i32, [vp, u64, i32, C.POINTER(C.c_double)]),
            "hnsw_server_get_stats": (i32, [vp, C.POINTER(ServerStats)]),
            "hnsw_server_cancel": (i32, [vp, u64]),
            "hnsw_server_destroy": (i32, [vp]),
            "hnsw_server_replay": (i32, [vp, C.POINTER(Request), vp, i64, i32, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int) -> None:
    if st != 0:
        raise HnswError(st, lib().hnsw_last_error().decode(errors="replace"))


def _ptr(x):
    """(address, keepalive) of a numpy array or torch tensor."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("buffer must be C-contiguous")
        return x.ctypes.data, x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), x
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def build_graph(data: np.ndarray, level_u: np.ndarray, metric: int = L2SQ, M: int = 16, Mmax: int | None = None,
                Mmax0: int | None = None, ef_construction: int = 200, mL: float | None = None,
                heuristic: bool = True, extend_candidates: bool = False, keep_pruned: bool = False,
                n_threads: int = 0) -> bytes:
    """Multi-threaded host construction (Alg. 1 + Alg. 4); returns an HNSWGB01 blob."""
    data = np.ascontiguousarray(data, dtype=np.float32)
    u = np.ascontiguousarray(level_u, dtype=np.float64)
    N, d = data.shape
    if u.shape != (N,):
        raise ValueError("level_u must hold one value per element")
    p = BuildParams(M, M if Mmax is None else Mmax, 2 * M if Mmax0 is None else Mmax0, ef_construction,
                    1.0 / np.log(M) if mL is None else mL, int(heuristic), int(extend_candidates),
                    int(keep_pruned), n_threads)
    out = C.c_void_p()
    nbytes = C.c_uint64()
    _check(lib().hnsw_build(data.ctypes.data, N, d, metric, C.byref(p), u.ctypes.data, C.byref(out),
                            C.byref(nbytes)))
    try:
        return C.string_at(out.value, nbytes.value)
    finally:
        lib().hnsw_free_blob(out)


def save_graph(blob: bytes, path: str) -> None:
    """hnsw_save_blob: validates the blob and writes it to `path`."""
    buf = np.frombuffer(blob, dtype=np.uint8)
    _check(lib().hnsw_save_blob(buf.ctypes.data, buf.size, os.fsencode(path)))


def load_graph(path: str) -> bytes:
    """hnsw_load_blob: reads and validates a graph file."""
    out = C.c_void_p()
    nbytes = C.c_uint64()
    _check(lib().hnsw_load_blob(os.fsencode(path), C.byref(out), C.byref(nbytes)))
    try:
        return C.string_at(out.value, nbytes.value)
    finally:
        lib().hnsw_free_blob(out)


def build_graph_gpu(data: np.ndarray, level_u: np.ndarray, metric: int = L2SQ, M: int = 16,
                    Mmax: int | None = None, Mmax0: int | None = None, ef_construction: int = 200,
                    mL: float | None = None, heuristic: bool = True, keep_pruned: bool = False,
                    n_threads: int = 0, stream=None) -> bytes:
    """hnsw_build_gpu: the seed (elements of level >= 1 and the first 4,096)
    built on the host, the other elements inserted into layer 0 on the current
    CUDA device in batches; returns an HNSWGB01 blob."""
    data = np.ascontiguousarray(data, dtype=np.float32)
    u = np.ascontiguousarray(level_u, dtype=np.float64)
    N, d = data.shape
    if u.shape != (N,):
        raise ValueError("level_u must hold one value per element")
    p = BuildParams(M, M if Mmax is None else Mmax, 2 * M if Mmax0 is None else Mmax0, ef_construction,
                    1.0 / np.log(M) if mL is None else mL, int(heuristic), 0, int(keep_pruned), n_threads)
    out = C.c_void_p()
    nbytes = C.c_uint64()
    _check(lib().hnsw_build_gpu(data.ctypes.data, N, d, metric, C.byref(p), u.ctypes.data, _stream_ptr(stream),
                                C.byref(out), C.byref(nbytes)))
    try:
        return C.string_at(out.value, nbytes.value)
    finally:
        lib().hnsw_free_blob(out)


class Index:
    """A graph resident on the current CUDA device."""

    def __init__(self, blob: bytes, storage: str | int = "f32", keep_fp32: bool = False, stream=None):
        st = DTYPES[storage] if isinstance(storage, str) else int(storage)
        buf = np.frombuffer(blob, dtype=np.uint8)
        h = C.c_void_p()
        _check(lib().hnsw_upload_index(buf.ctypes.data, buf.size, st, int(keep_fp32), _stream_ptr(stream),
                                       C.byref(h)))
        self.h = h
        self.info = IndexInfo()
        _check(lib().hnsw_get_index_info(self.h, C.byref(self.info)))

    def close(self) -> None:
        if getattr(self, "h", None) is not None and self.h.value:
            lib().hnsw_free_index(self.h)
            self.h = None

    def _refresh(self) -> None:
        _check(lib().hnsw_get_index_info(self.h, C.byref(self.info)))

    def debug_hold_decisions(self, on: bool) -> None:
        """hnsw_debug_hold_decisions (test hook): while on, the deferral's
        bounded wait runs out and the search reports ETIMEOUT."""
        _check(lib().hnsw_debug_hold_decisions(self.h, int(bool(on))))

    def reserve(self, capacity: int, stream=None) -> None:
        """hnsw_reserve: room for `capacity` elements (incremental insertion)."""
        _check(lib().hnsw_reserve(self.h, int(capacity), _stream_ptr(stream)))
        self._refresh()

    def insert(self, data, level_u, stream=None) -> range:
        """hnsw_insert: appends the rows of `data` (numpy array or CUDA tensor
        [n][d]) as new elements; returns their ids.  While searches run on
        other streams, pass a stream of its own (torch.cuda.Stream()): the
        legacy default stream would serialise them behind the insertion."""
        if isinstance(data, np.ndarray):
            data = np.ascontiguousarray(data, dtype=np.float32)
        u = np.ascontiguousarray(level_u, dtype=np.float64)
        n = int(data.shape[0])
        if u.shape != (n,):
            raise ValueError("level_u must hold one value per row")
        first = int(self.info.N)
        dp, _keep = _ptr(data)
        _check(lib().hnsw_insert(self.h, dp, n, u.ctypes.data, _stream_ptr(stream)))
        self._refresh()
        return range(first, first + n)

    def to_blob(self) -> bytes:
        """hnsw_index_to_blob: the current graph as an HNSWGB01 blob."""
        out = C.c_void_p()
        nbytes = C.c_uint64()
        _check(lib().hnsw_index_to_blob(self.h, C.byref(out), C.byref(nbytes)))
        try:
            return C.string_at(out.value, nbytes.value)
        finally:
            lib().hnsw_free_blob(out)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def d(self) -> int:
        return int(self.info.d)

    def set_stop_model(self, norm12, w_fp16) -> None:
        """Installs the learned-stop network (norm: mean[6], std[6]; 4,673 fp16 weights)."""
        norm = np.ascontiguousarray(norm12, dtype=np.float32)
        w = np.ascontiguousarray(w_fp16, dtype=np.float16).view(np.uint16)
        if norm.size != 12 or w.size != STOP_NPARAM:
            raise ValueError("norm needs 12 values, weights 4673")
        _check(lib().hnsw_set_stop_model(self.h, norm.ctypes.data, w.ctypes.data))

    def clear_stop_model(self) -> None:
        _check(lib().hnsw_clear_stop_model(self.h))

    def search_trace(self, queries, k: int, ef: int, max_checks: int, period: int = 4, logits: bool = False,
                     rerank: bool = False, visited_log2: int = 0, stream=None):
        """hnsw_search_trace on CUDA tensors; returns (feats, topk, logits|None,
        n_checks, ids, dists, stats) as CUDA tensors."""
        import torch
        n = queries.shape[0]
        dev = queries.device
        feats = torch.zeros((n, max_checks, 6), dtype=torch.float32, device=dev)
        topk = torch.zeros((n, max_checks, k), dtype=torch.int32, device=dev)
        lg = torch.zeros((n, max_checks), dtype=torch.float32, device=dev) if logits else None
        cnt = torch.zeros((n,), dtype=torch.int32, device=dev)
        ids = torch.empty((n, k), dtype=torch.int32, device=dev)
        ds = torch.empty((n, k), dtype=torch.float32, device=dev)
        st = torch.empty((n, 4), dtype=torch.int32, device=dev)
        p = SearchParams(k, ef, int(rerank), visited_log2, 2.0, period)
        _check(lib().hnsw_search_trace(self.h, C.byref(p), queries.data_ptr(), n, max_checks, feats.data_ptr(),
                                       topk.data_ptr(), lg.data_ptr() if lg is not None else None, cnt.data_ptr(),
                                       ids.data_ptr(), ds.data_ptr(), st.data_ptr(), _stream_ptr(stream)))
        return feats, topk, lg, cnt, ids, ds, st

    def search_into(self, queries, k: int, ef: int, out_ids, out_dists, stats=None, rerank: bool = False,
                    visited_log2: int = 0, stop_threshold: float = 2.0, stop_period: int = 0,
                    schedule: int = 0, stream=None, check_bounds: bool = False) -> None:
        """hnsw_search_ex into caller-owned buffers (host or device)."""
        n = int(queries.shape[0]) if queries is not None else 0
        p = SearchParams(k, ef, int(rerank), visited_log2, stop_threshold, stop_period, schedule,
                         int(check_bounds))
        qp, _a = _ptr(queries)
        ip, _b = _ptr(out_ids)
        dp, _c = _ptr(out_dists)
        sp, _d = _ptr(stats)
        _check(lib().hnsw_search_ex(self.h, C.byref(p), qp, n, ip, dp, sp, _stream_ptr(stream)))

    def search(self, queries, k: int, ef: int, rerank: bool = False, stats: bool = False, visited_log2: int = 0,
               stop_threshold: float = 2.0, stop_period: int = 0, schedule: int = 0, stream=None,
               check_bounds: bool = False):
        """Returns (ids, dists[, stats]) as arrays/tensors on the queries' device."""
        if hasattr(queries, "is_cuda") and queries.is_cuda:
            import torch
            n = queries.shape[0]
            ids = torch.empty((n, k), dtype=torch.int32, device=queries.device)
            ds = torch.empty((n, k), dtype=torch.float32, device=queries.device)
            st = torch.empty((n, 4), dtype=torch.int32, device=queries.device) if stats else None
        else:
            queries = np.ascontiguousarray(queries, dtype=np.float32)
            n = queries.shape[0]
            ids = np.empty((n, k), dtype=np.uint32)
            ds = np.empty((n, k), dtype=np.float32)
            st = np.empty((n, 4), dtype=np.uint32) if stats else None
        self.search_into(queries, k, ef, ids, ds, st, rerank=rerank, visited_log2=visited_log2,
                         stop_threshold=stop_threshold, stop_period=stop_period, schedule=schedule, stream=stream,
                         check_bounds=check_bounds)
        return (ids, ds, st) if stats else (ids, ds)


def merge_topk(shard_ids, shard_dists, id_base, k: int, stream=None):
    """hnsw_merge_topk: per-shard results [S][n][k] (CUDA tensors, local ids)
    -> the k smallest (distance, global id) over the shards, ([n][k] int32
    ids viewed as uint32, [n][k] float32), on the tensors' device."""
    import torch
    S, n, kk = shard_ids.shape
    if kk != k or tuple(shard_dists.shape) != (S, n, k):
        raise ValueError("shard results must be [S][n][k]")
    base = np.ascontiguousarray(id_base, dtype=np.uint32)
    if base.shape != (S,):
        raise ValueError("one id base per shard")
    si = shard_ids.contiguous()
    sd = shard_dists.contiguous()
    oi = torch.empty((n, k), dtype=torch.int32, device=si.device)
    od = torch.empty((n, k), dtype=torch.float32, device=si.device)
    _check(lib().hnsw_merge_topk(si.data_ptr(), sd.data_ptr(), S, base.ctypes.data, n, k, oi.data_ptr(),
                                 od.data_ptr(), _stream_ptr(stream)))
    return oi, od


def stop_grad(x, y, norm12, w_fp16):
    """hnsw_stop_grad: x [n,6] and y [n] CUDA float tensors; returns (grad[4673], loss)."""
    norm = np.ascontiguousarray(norm12, dtype=np.float32)
    w = np.ascontiguousarray(w_fp16, dtype=np.float16).view(np.uint16)
    g = np.zeros(STOP_NPARAM, dtype=np.float32)
    loss = C.c_float(0)
    _check(lib().hnsw_stop_grad(x.data_ptr(), y.data_ptr(), x.shape[0], norm.ctypes.data, w.ctypes.data,
                                g.ctypes.data, C.addressof(loss), _stream_ptr(None)))
    return g, float(loss.value)


def stop_train(x, y, w_init, epochs: int = 20, batch: int = 4096, lr: float = 2e-3, weight_decay: float = 0.0,
               seed: int = 0):
    """hnsw_stop_train on CUDA tensors x [n,6], y [n]; returns (norm12, w_fp16, loss_per_epoch)."""
    w0 = np.ascontiguousarray(w_init, dtype=np.float16).view(np.uint16)
    norm = np.zeros(12, dtype=np.float32)
    w = np.zeros(STOP_NPARAM, dtype=np.uint16)
    ls = np.zeros(epochs, dtype=np.float32)
    p = StopTrainParams(epochs, batch, lr, 0.0, 0.0, 0.0, weight_decay, seed)
    _check(lib().hnsw_stop_train(x.data_ptr(), y.data_ptr(), x.shape[0], C.byref(p), w0.ctypes.data,
                                 norm.ctypes.data, w.ctypes.data, ls.ctypes.data, _stream_ptr(None)))
    return norm, w.view(np.float16), ls


class Server:
    """Continuous-batching request loop over resident indexes (hnsw_server_*).
    Query and result buffers are numpy arrays kept alive until wait()."""

    def __init__(self, n_slots: int = 8, memory_budget: int = 0):
        h = C.c_void_p()
        _check(lib().hnsw_server_create(C.byref(ServerParams(n_slots, memory_budget)), C.byref(h)))
        self.h = h
        self._live = {}

    def add_index(self, index: Index) -> int:
        i = C.c_int32()
        _check(lib().hnsw_server_add_index(self.h, index.h, C.byref(i)))
        return int(i.value)

    def submit(self, index_id: int, queries, k: int, ef: int, rerank: bool = False, stop_threshold: float = 2.0,
               stop_period: int = 0) -> int:
        q = np.ascontiguousarray(queries, dtype=np.float32)
        n = q.shape[0]
        ids = np.empty((n, k), dtype=np.uint32)
        ds = np.empty((n, k), dtype=np.float32)
        r = Request(index_id, n, k, ef, int(rerank), stop_threshold, stop_period, q.ctypes.data, ids.ctypes.data,
                    ds.ctypes.data)
        t = C.c_uint64()
        _check(lib().hnsw_server_submit(self.h, C.byref(r), C.byref(t)))
        self._live[int(t.value)] = (q, ids, ds)
        return int(t.value)

    def replay(self, plan, arrival_s, timeout_ms: int = 600_000):
        """Native trace replay: plan is a list of (index_id, queries, k, ef,
        rerank[, stop_threshold, stop_period]); returns (per-request (ids,
        dists), latency_ms, submit_s)."""
        n = len(plan)
        reqs = (Request * n)()
        keep = []
        for i, item in enumerate(plan):
            idx, q, k, ef, rr = item[:5]
            thr, period = (item[5], item[6]) if len(item) > 5 else (2.0, 0)
            q = np.ascontiguousarray(q, dtype=np.float32)
            ids = np.empty((q.shape[0], k), dtype=np.uint32)
            ds = np.empty((q.shape[0], k), dtype=np.float32)
            reqs[i] = Request(idx, q.shape[0], k, ef, int(rr), float(thr), int(period), q.ctypes.data,
                              ids.ctypes.data, ds.ctypes.data)
            keep.append((q, ids, ds))
        arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
        lat = np.zeros(n, dtype=np.float64)
        sub = np.zeros(n, dtype=np.float64)
        _check(lib().hnsw_server_replay(self.h, reqs, arr.ctypes.data, n, timeout_ms, lat.ctypes.data, sub.ctypes.data))
        return [(k2[1], k2[2]) for k2 in keep], lat, sub

    def cancel(self, ticket: int) -> None:
        """hnsw_server_cancel: removes a request still waiting for admission
        (its wait then raises ECANCELED); EBUSY once it is admitted."""
        _check(lib().hnsw_server_cancel(self.h, ticket))

    def poll(self, ticket: int) -> bool:
        d = C.c_int32()
        _check(lib().hnsw_server_poll(self.h, ticket, C.byref(d)))
        return bool(d.value)

    def wait(self, ticket: int, timeout_ms: int = -1):
        """Returns (ids, dists, latency_ms) of a completed request."""
        lat = C.c_double()
        st = lib().hnsw_server_wait(self.h, ticket, timeout_ms, C.byref(lat))
        if st != 0 and st != 5:
            self._live.pop(ticket, None)
        _check(st)
        q, ids, ds = self._live.pop(ticket)
        return ids, ds, float(lat.value)

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().hnsw_server_get_stats(self.h, C.byref(s)))
        return {f: int(getattr(s, f)) for f, _ in ServerStats._fields_}

    def close(self) -> None:
        if getattr(self, "h", None) is not None and self.h.value:
            lib().hnsw_server_destroy(self.h)
            self.h = None
        self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
