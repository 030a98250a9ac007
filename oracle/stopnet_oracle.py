"""ORACLE of the learned early-stop network (test infrastructure only).

The paper has no learned component; this network is an addition beside the
plain method.  Definition (written here from the mathematics, in fp64):

  inputs   x in R^6 (search-state features), normalised x' = (x - mu) / sigma
  hidden   h1 = relu(W1 x' + b1)            W1: 64 x 6
           h2 = relu(W2 h1 + b2)            W2: 64 x 64
  output   z  = w3 . h2 + b3                 (logit of "stopping now loses nothing")
  loss     binary cross-entropy of sigmoid(z) against y in {0,1}, averaged
           over the batch:  l = max(z,0) - z y + log(1 + exp(-|z|))

Parameter vector (4,673 values, the order the library uses):
  W1 (row-major, out x in) | b1 | W2 (row-major, out x in) | b2 | w3 | b3

Features at a check step of the layer-0 beam (d1 = distance of the element
where the upper-layer descent ended, clamped below by 1e-12):
  0 log1p(best / d1)      best = nearest entry of W
  1 log1p(worst / d1)     worst = furthest entry of W
  2 log1p(n_eval)         distance evaluations so far
  3 log1p(d1)
  4 log1p(stale)          expansions since the K-th best entry last improved
  5 log1p(kth / d1)       K-th best entry of W
(ratios below 0 are clamped to 0).
"""
from __future__ import annotations

import numpy as np

NIN, NH = 6, 64
SIZES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta: np.ndarray) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def forward(theta, X, mu, sigma):
    """Returns the logits z[n] and the intermediates of the forward pass."""
    p = unpack(theta)
    Xn = (np.asarray(X, np.float64) - np.asarray(mu, np.float64)) / np.asarray(sigma, np.float64)
    a1 = Xn @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["w3"] + p["b3"][0]
    return z, (Xn, a1, h1, a2, h2)


def loss(theta, X, y, mu, sigma) -> float:
    z, _ = forward(theta, X, mu, sigma)
    y = np.asarray(y, np.float64)
    l = np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))
    return float(l.mean())


def grad(theta, X, y, mu, sigma) -> np.ndarray:
    """Gradient of the mean loss with respect to the parameter vector
    (chain rule through the layers above)."""
    p = unpack(theta)
    z, (Xn, a1, h1, a2, h2) = forward(theta, X, mu, sigma)
    n = z.shape[0]
    y = np.asarray(y, np.float64)
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / n          # d loss / d z
    g = {"w3": h2.T @ dz, "b3": np.array([dz.sum()])}
    da2 = np.outer(dz, p["w3"]) * (a2 > 0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    da1 = (da2 @ p["W2"]) * (a1 > 0)
    g["W1"] = da1.T @ Xn
    g["b1"] = da1.sum(0)
    return pack(g)


def features(best, worst, n_eval, d1, stale, kth):
    """The six features of one check step (see the module docstring)."""
    d = max(float(d1), 1e-12)
    return np.array([np.log1p(max(best / d, 0.0)), np.log1p(max(worst / d, 0.0)), np.log1p(n_eval),
                     np.log1p(max(d1, 0.0)), np.log1p(stale), np.log1p(max(kth / d, 0.0))])
