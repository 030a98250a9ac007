"""Seeded graphs shared by the tests, built by the ORACLE (never by the CUDA
library), cached per process."""
import functools

import numpy as np

from paper_1603_09320_gb300 import synth


@functools.lru_cache(maxsize=None)
def oracle_graph(name: str, n: int):
    from oracle import oracle as O
    p = synth.params(name)
    X = synth.base(name, n)
    g = O.Graph.build(X, synth.level_uniforms(name, n), **p)
    return g, X, g.to_blob()


def recall(ids, gt):
    k = gt.shape[1]
    return float(np.mean([len(set(ids[i][:k].tolist()) & set(gt[i].tolist())) / k for i in range(len(gt))]))
