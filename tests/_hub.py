"""A seeded input whose batched construction sends more than 256 new links to
one element in one batch (input generation only; no step of the method).

Integer coordinates in d = 16 (every fp32 distance exact).  Element 0, the
hub, sits at c = (100, ..., 100); elements 1 .. n_seed + n_fill - 1 are
fillers drawn uniformly from the integer box [180, 255]^16, far from c; the
last RAYS elements lie on rays from the hub along coordinate axes:
c + t e_k for k = 0..9, t = 1..30 (id = first + 30 k + t - 1), then one
point c + 40 e_10 (the last id).  Level draws: u = 1e-3 for the hub (level 3
with M = 8), u = 1 (level 0) for everything else, so the hub is the enter
point and the only element above layer 0.

With the first 4,096 elements as the seed and the growing batch schedule
(batches of max(64, inserted / 16)), three filler batches of 256, 272 and 289
follow the seed and the 301 ray points form the fourth batch.
"""
import numpy as np

D = 16
HUB = 100
N_SEED = 4096
FILL_BATCHES = (256, 272, 289)
RAYS = 10 * 30 + 1
PARAMS = dict(M=8, Mmax=8, Mmax0=16, efC=64)


def ray_ids(n_total: int):
    first = n_total - RAYS
    near = [first + 30 * k for k in range(10)]  # t = 1 on rays 0..9
    return first, near, n_total - 1             # the point at t = 40 on ray 10


def hub_input(seed: int = 7):
    rng = np.random.default_rng(seed)
    n_fill = N_SEED - 1 + sum(FILL_BATCHES)
    X = np.empty((1 + n_fill + RAYS, D), np.float32)
    X[0] = HUB
    X[1:1 + n_fill] = rng.integers(180, 256, size=(n_fill, D))
    r = 1 + n_fill
    for k in range(10):
        for t in range(1, 31):
            X[r] = HUB
            X[r, k] = HUB + t
            r += 1
    X[r] = HUB
    X[r, 10] = HUB + 40
    u = np.ones(X.shape[0])
    u[0] = 1e-3
    return X, u
