"""Cached construction of the synthetic workloads' graphs with the
multi-threaded host builder (Alg. 1 + Alg. 4).

The blob is kept under the system temp directory, keyed by the workload,
its size, the construction parameters and the builder's source, so a bench
and a test in the same machine build a 1M-element graph once.
"""
from __future__ import annotations

import hashlib
import os
import tempfile
import time

from . import hnsw, synth

CACHE = os.path.join(tempfile.gettempdir(), "hnsw_gb300_cache")
_HERE = os.path.dirname(os.path.abspath(__file__))


def build_or_load(name: str, n: int, threads: int = 0, X=None, log=None):
    """Returns (blob, seconds spent building or None when loaded)."""
    p = synth.params(name)
    src = open(os.path.join(_HERE, "csrc", "builder.cpp"), "rb").read()
    key = hashlib.sha256(repr((name, n, p, hashlib.sha256(src).hexdigest())).encode()).hexdigest()[:16]
    os.makedirs(CACHE, exist_ok=True)
    path = os.path.join(CACHE, f"{name}_{n}_{key}.blob")
    if os.path.exists(path):
        with open(path, "rb") as f:
            return f.read(), None
    if X is None:
        X = synth.base(name, n)
    u = synth.level_uniforms(name, n)
    t = time.time()
    blob = hnsw.build_graph(X, u, metric=p["metric"], M=p["M"], Mmax=p["Mmax"], Mmax0=p["Mmax0"],
                            ef_construction=p["efC"], n_threads=threads)
    dt = time.time() - t
    if log:
        log(f"built {name} graph N={n} in {dt:.1f}s")
    tmp = path + f".{os.getpid()}"
    with open(tmp, "wb") as f:
        f.write(blob)
    os.replace(tmp, path)
    return blob, dt
