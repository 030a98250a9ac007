"""Host side of the learned stop's training pipeline (no GPU): the label of a
check step, worked out by hand, and the initial weights' layout."""
import numpy as np

from paper_1603_09320_gb300 import stopnet


def test_labels_by_hand():
    # two queries, k = 2, up to three checks each; exact neighbours {1, 2} and {5, 6}
    gt = np.array([[1, 2], [5, 6]])
    final = np.array([[1, 9], [5, 6]])  # the fixed-ef result finds 1 and 2 of them
    topk = np.array([[[7, 8], [1, 8], [2, 3]],
                     [[5, 7], [6, 5], [0, 0]]])
    n_checks = np.array([3, 2])
    mask, y = stopnet.labels_from_trace(topk, n_checks, final, gt)
    assert mask.tolist() == [[True, True, True], [True, True, False]]
    # query 0 needs one true neighbour (as many as its final result), query 1 two
    assert y.tolist() == [[0.0, 1.0, 1.0], [0.0, 1.0, 0.0]]


def test_initial_weights_layout():
    w = stopnet.init_weights(3)
    assert w.dtype == np.float16 and w.size == 6 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 4673
    b1 = w[384:448]
    b2 = w[448 + 4096:448 + 4096 + 64]
    assert not b1.any() and not b2.any() and w[-1] == 0
    assert np.array_equal(w, stopnet.init_weights(3)) and not np.array_equal(w, stopnet.init_weights(4))
    w1 = w[:384].astype(np.float64)
    assert abs(w1.std() - np.sqrt(2.0 / 6)) < 0.1  # He-normal fan-in 6
