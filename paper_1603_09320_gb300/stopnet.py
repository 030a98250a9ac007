"""Training pipeline of the learned early stop (an addition; the paper has
none): initial weights, labels from search traces, and the (ef, threshold)
choice.

Label of a check step (the search state every `period` layer-0 expansions of
a search run at a fixed ef): 1 when the top-k of W at that step already holds
at least as many true nearest neighbours (exact fp64 k-NN) as the final
result of that same fixed-ef search, i.e. stopping there loses no recall
against the fixed-ef method; else 0.  All arithmetic of the network itself
runs in the library's CUDA kernels.
"""
from __future__ import annotations

import numpy as np

from . import hnsw, synth

NIN, NH = 6, 64


def init_weights(seed: int = 0) -> np.ndarray:
    """He-normal weights (zero biases, small output layer) as fp16, drawn by
    the seeded counter-based generator."""
    r = synth.rng(seed)
    w1 = r.normal(0, np.sqrt(2.0 / NIN), size=(NH, NIN))
    w2 = r.normal(0, np.sqrt(2.0 / NH), size=(NH, NH))
    w3 = r.normal(0, np.sqrt(1.0 / NH), size=NH)
    theta = np.concatenate([w1.ravel(), np.zeros(NH), w2.ravel(), np.zeros(NH), w3, [0.0]])
    return theta.astype(np.float16)


def labels_from_trace(topk: np.ndarray, n_checks: np.ndarray, final_ids: np.ndarray, gt: np.ndarray):
    """(X-row mask, labels) for the recorded checks.  topk [n][C][k],
    n_checks [n], final_ids [n][k], gt [n][k] exact neighbours."""
    n, cmax, k = topk.shape
    gts = [set(g.tolist()) for g in gt]
    final_hits = np.array([len(set(final_ids[i].tolist()) & gts[i]) for i in range(n)])
    mask = np.arange(cmax)[None, :] < n_checks[:, None]
    y = np.zeros((n, cmax), dtype=np.float32)
    for i in range(n):
        for c in range(int(n_checks[i])):
            y[i, c] = 1.0 if len(set(topk[i, c].tolist()) & gts[i]) >= final_hits[i] else 0.0
    return mask, y


def train_from_trace(feats, mask, y, epochs: int = 30, batch: int = 4096, lr: float = 2e-3, seed: int = 0):
    """Trains on the GPU (hnsw_stop_train) on the masked check steps."""
    import torch
    X = torch.as_tensor(np.ascontiguousarray(feats[mask].reshape(-1, NIN), dtype=np.float32)).cuda()
    Y = torch.as_tensor(np.ascontiguousarray(y[mask].reshape(-1), dtype=np.float32)).cuda()
    return hnsw.stop_train(X, Y, init_weights(seed), epochs=epochs, batch=batch, lr=lr, seed=seed)
