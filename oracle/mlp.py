"""FP64 oracle of the learned-proposal network (TEST INFRASTRUCTURE; see oracle/__init__.py).

Plain NumPy restatement of the definitions, with no blocking or fusion:
  forward   a_0 = x;  a_l = relu(a_{l-1} W_l^T + b_l) for hidden layers;  z = a_{L-1} W_L^T + b_L
  loss      mean over rows of sum over bins of  max(z, 0) - y z + log(1 + exp(-|z|))
            (binary cross-entropy with logits, the numerically stable form of
             -[y log s(z) + (1 - y) log(1 - s(z))], s = logistic sigmoid)
  backward  dz = (s(z) - y) / B;  dW_l = dz_l^T a_{l-1};  db_l = sum_rows dz_l;
            da_{l-1} = dz_l W_l;  dz_{l-1} = da_{l-1} * [a_{l-1} > 0]
  Adam      (Kingma & Ba 2015) m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
            w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
Layer sizes are arguments, so the finite-difference pins can use tiny networks.
"""
from __future__ import annotations

import numpy as np


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(params, x):
    """params: list of (W (out x in), b (out,)). Returns (logits, activations list incl. input)."""
    acts = [np.asarray(x, np.float64)]
    a = acts[0]
    for i, (W, b) in enumerate(params):
        z = a @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        if i < len(params) - 1:
            a = np.maximum(z, 0.0)
            acts.append(a)
        else:
            return z, acts
    raise ValueError("empty network")


def bce_with_logits(z, y):
    """Mean over rows of the summed per-bin binary cross-entropy."""
    per = np.maximum(z, 0.0) - y * z + np.log1p(np.exp(-np.abs(z)))
    return float(np.sum(per) / z.shape[0])


def loss_and_grads(params, x, y):
    z, acts = forward(params, x)
    B = z.shape[0]
    loss = bce_with_logits(z, y)
    dz = (sigmoid(z) - y) / B
    grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        W = np.asarray(params[i][0], np.float64)
        grads[i] = (dz.T @ acts[i], dz.sum(axis=0))
        if i > 0:
            da = dz @ W
            dz = da * (acts[i] > 0)
    return loss, grads


def adam(w, m, v, g, lr, b1, b2, eps, t):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    w = w - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return w, m, v
