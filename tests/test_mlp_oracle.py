"""Pins of the FP64 network oracle: finite differences, closed forms (CPU only)."""
import math

import numpy as np

from oracle import mlp


def _net(rng, sizes):
    return [(rng.standard_normal((o, i)) / math.sqrt(i), rng.standard_normal(o) * 0.1)
            for i, o in zip(sizes[:-1], sizes[1:])]


def test_bce_closed_forms():
    z = np.array([[0.0, 2.0, -3.0]])
    y = np.array([[1.0, 0.0, 1.0]])
    expect = math.log(2.0) + math.log(1 + math.exp(2.0)) + math.log(1 + math.exp(3.0))
    assert abs(mlp.bce_with_logits(z, y) - expect) < 1e-12
    # large logits stay finite and exact
    assert abs(mlp.bce_with_logits(np.array([[800.0]]), np.array([[0.0]])) - 800.0) < 1e-9


def test_forward_relu_and_affine_by_hand():
    W1 = np.array([[1.0, -1.0], [2.0, 0.5]])
    b1 = np.array([0.0, -1.0])
    W2 = np.array([[1.0, 1.0]])
    b2 = np.array([0.25])
    x = np.array([[1.0, 3.0]])
    # hidden = relu([1 - 3, 2 + 1.5 - 1]) = [0, 2.5]; z = 2.5 + 0.25
    z, acts = mlp.forward([(W1, b1), (W2, b2)], x)
    assert z.shape == (1, 1) and abs(z[0, 0] - 2.75) < 1e-15
    np.testing.assert_array_equal(acts[1], [[0.0, 2.5]])


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    sizes = [6, 5, 4, 3]
    params = _net(rng, sizes)
    x = rng.standard_normal((7, sizes[0]))
    y = (rng.random((7, sizes[-1])) < 0.3).astype(np.float64)
    _, grads = mlp.loss_and_grads(params, x, y)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            num = np.zeros_like(arr)
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + h
                lp = mlp.bce_with_logits(mlp.forward(params, x)[0], y)
                arr[idx] = old - h
                lm = mlp.bce_with_logits(mlp.forward(params, x)[0], y)
                arr[idx] = old
                num[idx] = (lp - lm) / (2 * h)
            rel = np.linalg.norm(num - g) / max(np.linalg.norm(g), 1e-30)
            assert rel < 1e-6, (li, rel)


def test_adam_first_step_is_sign_step():
    """At t = 1 with zero moments, Adam moves every weight by lr * g / (|g| + eps')."""
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    w1, m, v = mlp.adam(w, np.zeros(3), np.zeros(3), g, 0.01, 0.9, 0.999, 1e-8, 1)
    np.testing.assert_allclose(w1, w - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
