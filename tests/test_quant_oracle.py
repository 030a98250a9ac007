"""Pins of the storage-form oracle (oracle/quant_oracle.py) on the CPU: each
number format against a library conversion of the same format and against
values worked out by hand from its definition."""
import numpy as np
import pytest

from oracle import quant_oracle as QO

torch = pytest.importorskip("torch")


def torch_e4m3(v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).to(torch.float8_e4m3fn).view(torch.uint8).numpy()


def test_e4m3_magnitudes_by_hand():
    m = QO.e4m3_magnitudes()
    assert len(m) == 127 and np.all(np.diff(m) > 0)
    assert m[0] == 0.0 and m[1] == 2.0 ** -9  # smallest subnormal
    assert m[7] == 7 / 8 * 2.0 ** -6 and m[8] == 2.0 ** -6  # largest subnormal, smallest normal
    assert m[0x38] == 1.0 and m[0x39] == 1.125
    assert m[126] == 448.0 and m[125] == 416.0


def test_e4m3_encode_hand_values():
    cases = [
        (448.0, 0x7E), (1000.0, 0x7E), (-1000.0, 0xFE), (460.0, 0x7E),  # saturation
        (2.0 ** -9, 0x01), (2.0 ** -10, 0x00),  # half the smallest subnormal: tie to even (0)
        (3 * 2.0 ** -10, 0x02),  # between codes 1 and 2: tie to even
        (1.0625, 0x38),  # between 1 (0x38) and 1.125 (0x39): tie to even
        (1.1875, 0x3A),  # between 1.125 (0x39) and 1.25 (0x3A): tie to even
        (1.07, 0x39), (1.05, 0x38), (-1.0, 0xB8), (0.0, 0x00), (-0.0, 0x80),
    ]
    v = np.array([c[0] for c in cases], dtype=np.float32)
    assert QO.e4m3_encode(v).tolist() == [c[1] for c in cases]


def test_e4m3_encode_matches_torch_cast():
    rng = np.random.default_rng(11)
    m = QO.e4m3_magnitudes()
    mids = ((m[:-1] + m[1:]) / 2).astype(np.float32)  # every tie (exact in fp32)
    assert np.all(mids.astype(np.float64) == (m[:-1] + m[1:]) / 2)
    scale = rng.choice([1e-4, 1e-2, 1.0, 30.0, 200.0], 100_000)
    rnd = np.clip(rng.standard_normal(100_000) * scale, -448, 448).astype(np.float32)
    v = np.concatenate([mids, -mids, m.astype(np.float32), rnd])
    np.testing.assert_array_equal(QO.e4m3_encode(v), torch_e4m3(v))
    # decode(encode(v)) is the nearest magnitude: no code is closer
    dec = QO.e4m3_decode(QO.e4m3_encode(rnd))
    best = np.abs(np.abs(rnd.astype(np.float64))[:, None] - m[None, :]).min(axis=1)
    np.testing.assert_array_equal(np.abs(np.abs(rnd) - np.abs(dec)), best)


def test_bf16_round_by_hand_and_against_torch():
    one = 1.0
    cases = [(one + 2.0 ** -8, 1.0),  # tie, even neighbour below
             (one + 3 * 2.0 ** -8, one + 2.0 ** -6),  # tie, odd neighbour below: up
             (one + 2.0 ** -8 + 2.0 ** -20, one + 2.0 ** -7),  # above the tie
             (-(one + 2.0 ** -8), -1.0), (3.0, 3.0)]
    v = np.array([c[0] for c in cases], dtype=np.float32)
    np.testing.assert_array_equal(QO.bf16_round(v), np.array([c[1] for c in cases], dtype=np.float32))
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(200_000) * np.exp(rng.uniform(-40, 40, 200_000))).astype(np.float32)
    ties = ((rng.integers(0, 1 << 16, 5000, dtype=np.uint64) << 16) | 0x8000).astype(np.uint32).view(np.float32)
    ties = ties[np.isfinite(ties)]
    x = np.concatenate([x, ties])
    ref = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    np.testing.assert_array_equal(QO.bf16_round(x).view(np.uint32), ref.view(np.uint32))


def test_f16_round_by_hand_and_against_torch():
    cases = [(1.0 + 2.0 ** -11, 1.0), (1.0 + 3 * 2.0 ** -11, 1.0 + 2.0 ** -9), (65519.0, 65504.0),
             (2.0 ** -24, 2.0 ** -24), (2.0 ** -25, 0.0)]
    v = np.array([c[0] for c in cases], dtype=np.float32)
    np.testing.assert_array_equal(QO.f16_round(v), np.array([c[1] for c in cases], dtype=np.float32))
    x = np.random.default_rng(6).uniform(-2, 2, 100_000).astype(np.float32)
    ref = torch.from_numpy(x).half().float().numpy()
    np.testing.assert_array_equal(QO.f16_round(x), ref)


def test_fp8_rows_scale_and_error_bound():
    rng = np.random.default_rng(7)
    X = (rng.standard_normal((500, 100)) * rng.uniform(0.01, 50, (500, 1))).astype(np.float32)
    X[3] = 0.0
    codes, s = QO.fp8_rows(X)
    assert s[3] == 1.0 and not codes[3].any()
    live = np.arange(500) != 3
    # s = max|x| / 448 in fp32, and the largest element encodes to +-448
    np.testing.assert_array_equal(s, np.where(live, np.abs(X).max(1) / np.float32(448), 1).astype(np.float32))
    amax = np.abs(X).argmax(1)
    assert np.all((codes[live, amax[live]] & 0x7F) == 126)
    # relative error of a normal-range element: at most half a step, 2^-4
    Y = QO.decoded_rows("fp8", X)
    normal = np.abs(X) >= 2.0 ** -6 * s[:, None] * 1.0001
    rel = np.abs(Y[normal].astype(np.float64) - X[normal]) / np.abs(X[normal])
    assert rel.max() <= 2.0 ** -4 * (1 + 1e-6)
    np.testing.assert_array_equal(np.sign(Y[normal]), np.sign(X[normal]))


def test_graph_with_data_keeps_every_link():
    from oracle import oracle as O
    from paper_1603_09320_gb300 import synth
    p = synth.params("tiny")
    X = synth.base("tiny", 2000)
    g = O.Graph.build(X, synth.level_uniforms("tiny", 2000), **p)
    Q = synth.queries("tiny", 30)
    same = g.with_data(X)
    for a, b in zip(g.knn_search_batch(Q, 10, 32), same.knn_search_batch(Q, 10, 32)):
        np.testing.assert_array_equal(a, b)
    Y = QO.decoded_rows("fp8", X)
    h = g.with_data(Y)
    assert h.enter_point == g.enter_point and np.array_equal(h.levels(), g.levels())
    for i in range(0, 2000, 37):
        assert h.neighbors(i, 0) == g.neighbors(i, 0)
    assert h.dist(Q[0], 5) == float(((Q[0].astype(np.float64) - Y[5]) ** 2).sum())
    with pytest.raises(ValueError):
        g.with_data(X[:10])
