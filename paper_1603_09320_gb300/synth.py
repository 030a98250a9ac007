"""Seeded synthetic workloads shaped like the paper's evaluation data.

This module only draws random numbers: it holds none of the method's
arithmetic, and both the CUDA library's tests/bench and the oracle take their
inputs from it.  The generator is numpy's Philox (a counter-based generator),
so every array is a pure function of (seed, shape).

Workloads (Section 5.2, Table 1 names the public datasets these stand in for;
the datasets themselves are not used):
  tiny    N=10,000  d=32  i.i.d. uniform integers 0..255 (as fp32), squared L2
  sift    N=1,000,000 d=128 integer coordinates 0..255 drawn from a mixture of
          1,000 Gaussian clusters (centres uniform in [0,255], per-cluster sigma
          uniform in [10,40], clipped and rounded), squared L2   (SIFT 1M shape)
  glove   N=1,200,000 d=100 unit vectors from a mixture of 500 Gaussian clusters
          with Zipf(1.1) weights, cosine distance               (GloVe shape)
  lowd    N=10,000,000 d=8: 95% from 10,000 tight clusters (sigma 1e-3) in
          [0,1]^8, 5% uniform background, squared L2             (random d=4..10)
Seeds: base data 1000+c, queries 2000+c, level draws 3000+c, training
queries 4000+c, where c is the workload's index (tiny 0, sift 1, glove 2, lowd 3).
"""
from __future__ import annotations

import numpy as np

WORKLOADS = {
    # name: (index, N, d, metric, M, Mmax, Mmax0, efC, n_queries)
    "tiny": (0, 10_000, 32, 0, 8, 8, 16, 64, 1_000),
    "sift": (1, 1_000_000, 128, 0, 16, 16, 32, 200, 10_000),
    "glove": (2, 1_200_000, 100, 1, 16, 16, 32, 500, 10_000),
    "lowd": (3, 10_000_000, 8, 0, 12, 12, 24, 100, 100_000),
}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=seed))


def uniform_open01(seed: int, n: int) -> np.ndarray:
    """n draws of u in (0, 1], 53-bit resolution: u = (x + 1) / 2**53."""
    x = rng(seed).integers(0, 2**53, size=n, dtype=np.int64)
    return (x.astype(np.float64) + 1.0) / float(2**53)


def _uniform_ints(seed: int, n: int, d: int) -> np.ndarray:
    return rng(seed).integers(0, 256, size=(n, d)).astype(np.float32)


class _SiftMixture:
    def __init__(self, d: int = 128, n_clusters: int = 1000, seed: int = 1001):
        r = rng(seed * 7919 + 17)
        self.centres = r.uniform(0.0, 255.0, size=(n_clusters, d)).astype(np.float32)
        self.sigma = r.uniform(10.0, 40.0, size=n_clusters).astype(np.float32)

    def draw(self, seed: int, n: int) -> np.ndarray:
        r = rng(seed)
        out = np.empty((n, self.centres.shape[1]), dtype=np.float32)
        step = 1 << 16
        for s in range(0, n, step):
            m = min(step, n - s)
            c = r.integers(0, self.centres.shape[0], size=m)
            z = r.standard_normal(size=(m, self.centres.shape[1]), dtype=np.float32)
            x = self.centres[c] + self.sigma[c, None] * z
            out[s:s + m] = np.rint(np.clip(x, 0.0, 255.0))
        return out


class _GloveMixture:
    def __init__(self, d: int = 100, n_clusters: int = 500, seed: int = 1002):
        r = rng(seed * 7919 + 17)
        self.centres = r.standard_normal(size=(n_clusters, d)).astype(np.float32)
        w = 1.0 / np.arange(1, n_clusters + 1, dtype=np.float64) ** 1.1
        self.cdf = np.cumsum(w / w.sum())

    def draw(self, seed: int, n: int) -> np.ndarray:
        r = rng(seed)
        out = np.empty((n, self.centres.shape[1]), dtype=np.float32)
        step = 1 << 16
        for s in range(0, n, step):
            m = min(step, n - s)
            c = np.minimum(np.searchsorted(self.cdf, r.random(m)), self.centres.shape[0] - 1)
            z = r.standard_normal(size=(m, self.centres.shape[1]), dtype=np.float32)
            x = self.centres[c] + np.float32(0.5) * z
            nrm = np.sqrt((x * x).sum(axis=1, dtype=np.float32))
            out[s:s + m] = x / nrm[:, None]
        return out


class _LowdMixture:
    def __init__(self, d: int = 8, n_clusters: int = 10_000, seed: int = 1003):
        r = rng(seed * 7919 + 17)
        self.centres = r.uniform(0.0, 1.0, size=(n_clusters, d)).astype(np.float32)

    def draw(self, seed: int, n: int, frac_cluster: float) -> np.ndarray:
        r = rng(seed)
        d = self.centres.shape[1]
        out = np.empty((n, d), dtype=np.float32)
        step = 1 << 18
        for s in range(0, n, step):
            m = min(step, n - s)
            from_cluster = r.random(m) < frac_cluster
            c = r.integers(0, self.centres.shape[0], size=m)
            x = self.centres[c] + np.float32(1e-3) * r.standard_normal(size=(m, d), dtype=np.float32)
            u = r.uniform(0.0, 1.0, size=(m, d)).astype(np.float32)
            out[s:s + m] = np.where(from_cluster[:, None], x, u)
        return out


def base(name: str, n: int | None = None) -> np.ndarray:
    """n base vectors of a workload (default: its full size).  Rows are drawn
    in chunks (65,536 rows; 262,144 for lowd), so the first whole chunks of a
    smaller draw equal those of the full-size one; the rows after the last
    whole chunk follow the same distribution but are other draws."""
    idx, N, d, *_ = WORKLOADS[name]
    n = N if n is None else n
    seed = 1000 + idx
    if name == "tiny":
        return _uniform_ints(seed, n, d)
    if name == "sift":
        return _SiftMixture(d, seed=seed).draw(seed, n)
    if name == "glove":
        return _GloveMixture(d, seed=seed).draw(seed, n)
    if name == "lowd":
        return _LowdMixture(d, seed=seed).draw(seed, n, 0.95)
    raise KeyError(name)


def queries(name: str, n: int | None = None, training: bool = False) -> np.ndarray:
    """Query vectors from the same distribution as the base (seed 2000+c, or
    4000+c for the training queries of the learned stop)."""
    idx, N, d, _m, _M, _a, _b, _e, nq = WORKLOADS[name]
    n = nq if n is None else n
    seed = (4000 if training else 2000) + idx
    if name == "tiny":
        return _uniform_ints(seed, n, d)
    if name == "sift":
        return _SiftMixture(d, seed=1000 + idx).draw(seed, n)
    if name == "glove":
        return _GloveMixture(d, seed=1000 + idx).draw(seed, n)
    if name == "lowd":
        return _LowdMixture(d, seed=1000 + idx).draw(seed, n, 0.90)
    raise KeyError(name)


def level_uniforms(name: str, n: int | None = None) -> np.ndarray:
    """The u of the level draw of Alg. 1 for elements 0..n-1 (seed 3000+c)."""
    idx, N, *_ = WORKLOADS[name]
    return uniform_open01(3000 + idx, N if n is None else n)


def params(name: str) -> dict:
    idx, N, d, metric, M, Mmax, Mmax0, efC, nq = WORKLOADS[name]
    return dict(metric=metric, M=M, Mmax=Mmax, Mmax0=Mmax0, efC=efC, mL=1.0 / np.log(M))
