"""Oracle pins for the density-reconstruction MLP: central finite differences
of the loss against the analytic gradient, softmax rows summing to 1, and an
Adam step against its closed form on a scalar."""
import numpy as np

import oracle


def _setup(seed=0):
    rng = np.random.default_rng(seed)
    sizes = [7, 9, 8, 5]
    params = oracle.mlp_init(sizes, rng)
    params = [(w, rng.normal(0, 0.1, b.shape)) for w, b in params]
    x = rng.normal(size=(6, 7))
    t = rng.random((6, 5))
    t /= t.sum(axis=1, keepdims=True)
    return params, x, t


def test_softmax_rows_are_distributions():
    params, x, _ = _setup()
    p, _, _ = oracle.mlp_forward(params, x)
    assert np.allclose(p.sum(axis=1), 1.0) and p.min() > 0


def test_gradient_matches_central_differences():
    params, x, t = _setup(1)
    loss, grads = oracle.mlp_loss_grad(params, x, t)
    h = 1e-6
    for l, (w, b) in enumerate(params):
        for arr, g in ((w, grads[l][0]), (b, grads[l][1])):
            flat = arr.reshape(-1)
            for idx in range(0, flat.size, max(1, flat.size // 7)):
                old = flat[idx]
                flat[idx] = old + h
                lp, _ = oracle.mlp_loss_grad(params, x, t)
                flat[idx] = old - h
                lm, _ = oracle.mlp_loss_grad(params, x, t)
                flat[idx] = old
                num = (lp - lm) / (2 * h)
                assert abs(num - g.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(num))


def test_cross_entropy_is_minimal_at_the_target():
    # with one linear layer and logits = log t, the loss equals the entropy of t
    t = np.array([[0.2, 0.3, 0.5]])
    params = [(np.zeros((3, 1)), np.log(t[0]))]
    loss, grads = oracle.mlp_loss_grad(params, np.ones((1, 1)), t)
    assert abs(loss - (-np.sum(t * np.log(t)))) < 1e-12
    assert np.abs(grads[0][1]).max() < 1e-12


def test_adam_first_step_is_lr_times_sign():
    # after one step from zero moments, the bias-corrected update is lr * g / (|g| + eps)
    params = [(np.array([[1.0]]), np.array([0.5]))]
    grads = [(np.array([[2.0]]), np.array([-3.0]))]
    zero = [(np.zeros((1, 1)), np.zeros(1))]
    p, m, v = oracle.adam_step(params, grads, zero, zero, 1, 0.01)
    assert abs(p[0][0][0, 0] - (1.0 - 0.01 * 2.0 / (2.0 + 1e-8))) < 1e-12
    assert abs(p[0][1][0] - (0.5 + 0.01 * 3.0 / (3.0 + 1e-8))) < 1e-12


def test_features_hand_example():
    # two bins with masses 0.25 / 0.75 -> densities 0.5 / 1.5; moments d_1 only
    x = oracle.mlp_features([[0.25, 0.75]], [[1.0, 0.5, 0.1]], 2)
    assert np.array_equal(x, [[0.5, 1.5, 0.5]])


def test_graph_stats_and_degree_features_hand_example():
    # degrees of the star K_{1,3}: 3, 1, 1, 1
    st = oracle.graph_stats([3, 1, 1, 1], 8)
    assert np.array_equal(st, [1.5, 3.0, 3.0, 32.0])
    x = oracle.mlp_features([[0.5, 0.5]], [[1.0, 0.2]], 2, stats=[st])
    want = [1.0, 1.0, 0.2, np.log(1.5) / 10, (0.5 * np.log(3.0) - np.log(1.5)) / 10, np.log(3.0) / 10,
            np.log(32.0) / 10]
    assert np.allclose(x, [want], rtol=0, atol=1e-15)
    # a regular graph has no degree spread
    x = oracle.mlp_features([[1.0]], [[1.0]], 1, stats=[oracle.graph_stats([4, 4, 4, 4, 4], 1)])
    assert abs(x[0, 2]) < 1e-15 and abs(x[0, 1] - np.log(4.0) / 10) < 1e-15


def test_normalize_hist_hand_example():
    t = oracle.normalize_hist([[-0.1, 0.3, 0.1], [-1.0, 0.0, -2.0]])
    assert np.allclose(t, [[0.0, 0.75, 0.25], [1 / 3, 1 / 3, 1 / 3]], rtol=0, atol=1e-15)
