"""The seeded input recipes (paper_1603_09320_gb300/synth.py) produce what
their descriptions state: shapes, value sets, cluster structure and mixture
weights, level draws in (0, 1], and the same arrays for the same seeds."""
import numpy as np

from paper_1603_09320_gb300 import synth


def test_shapes_params_and_determinism():
    for name, (idx, N, d, metric, M, Mmax, Mmax0, efC, nq) in synth.WORKLOADS.items():
        X = synth.base(name, 1000)
        assert X.shape == (1000, d) and X.dtype == np.float32
        assert np.array_equal(X, synth.base(name, 1000))
        Q = synth.queries(name, 50)
        assert Q.shape == (50, d) and not np.array_equal(Q, X[:50])
        T = synth.queries(name, 50, training=True)
        assert not np.array_equal(T, Q)
        p = synth.params(name)
        assert (p["M"], p["Mmax"], p["Mmax0"], p["efC"], p["metric"]) == (M, Mmax, Mmax0, efC, metric)
        assert p["Mmax0"] == 2 * p["M"] and abs(p["mL"] - 1.0 / np.log(M)) < 1e-15


def test_smaller_draws_share_whole_chunks():
    a = synth.base("sift", 70_000)
    b = synth.base("sift", 131_072)
    assert np.array_equal(a[:65_536], b[:65_536])


def test_level_uniforms_open_at_zero():
    u = synth.level_uniforms("sift", 200_000)
    assert u.min() > 0.0 and u.max() <= 1.0
    assert abs(u.mean() - 0.5) < 0.005
    assert np.array_equal(u[:1000], synth.level_uniforms("sift", 1000))  # one draw per element


def test_tiny_uniform_integers():
    X = synth.base("tiny", 10_000)
    assert np.array_equal(X, np.rint(X)) and X.min() == 0 and X.max() == 255
    counts = np.bincount(X.astype(np.int64).ravel(), minlength=256)
    assert counts.min() > 0.8 * X.size / 256 and counts.max() < 1.2 * X.size / 256


def test_sift_shaped_clusters():
    X = synth.base("sift", 20_000)
    assert np.array_equal(X, np.rint(X)) and X.min() >= 0 and X.max() <= 255
    mix = synth._SiftMixture(128, seed=1001)
    # every point lies near one of the 1,000 centres: distance to the nearest
    # centre ~ sigma * sqrt(d), sigma in [10, 40] (clipping only shortens it)
    c = mix.centres.astype(np.float64)
    x = X[:2000].astype(np.float64)
    d2 = (x * x).sum(1)[:, None] - 2 * x @ c.T + (c * c).sum(1)[None, :]
    near = np.sqrt(np.maximum(d2.min(1), 0))
    assert near.max() < 45 * np.sqrt(128) and np.median(near) > 9 * np.sqrt(128)
    # and much nearer than to a typical centre
    assert np.median(near) < 0.5 * np.median(np.sqrt(np.maximum(d2, 0)))


def test_glove_shaped_unit_vectors_with_zipf_weights():
    X = synth.base("glove", 30_000)
    np.testing.assert_allclose(np.linalg.norm(X.astype(np.float64), axis=1), 1.0, atol=1e-5)
    mix = synth._GloveMixture(100, seed=1002)
    c = mix.centres / np.linalg.norm(mix.centres, axis=1, keepdims=True)
    lab = np.argmax(X @ c.T, axis=1)  # clusters are well separated on the sphere
    share = np.bincount(lab, minlength=500) / len(X)
    w = 1.0 / np.arange(1, 501) ** 1.1
    w /= w.sum()
    assert abs(share[0] - w[0]) < 0.01 and abs(share[1] - w[1]) < 0.01
    assert abs(share[:10].sum() - w[:10].sum()) < 0.02


def test_lowd_clustered_fraction():
    mix = synth._LowdMixture(8, seed=1003)

    def clustered_fraction(Y):
        c = mix.centres.astype(np.float64)
        y = Y.astype(np.float64)
        best = np.full(len(y), np.inf)
        for s in range(0, len(c), 2000):
            cc = c[s:s + 2000]
            d2 = (y * y).sum(1)[:, None] - 2 * y @ cc.T + (cc * cc).sum(1)[None, :]
            best = np.minimum(best, d2.min(1))
        return np.mean(np.sqrt(np.maximum(best, 0)) < 8e-3)  # sigma 1e-3, d = 8: radius ~2.8e-3

    X = synth.base("lowd", 4000)
    assert X.min() >= -0.01 and X.max() <= 1.01
    assert abs(clustered_fraction(X) - 0.95) < 0.015
    assert abs(clustered_fraction(synth.queries("lowd", 4000)) - 0.90) < 0.02
