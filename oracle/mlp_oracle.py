"""Reference for the cost model's kernels: a one-hidden-layer ReLU perceptron
in float64 numpy (forward, mean squared error, gradient by the chain rule).

TEST INFRASTRUCTURE (part of the oracle; see ``oracle/__init__.py``). The
network is not part of the sorting method. Parameter layout as in
include/onesweep_mlp.h: W1 [hidden][features], b1 [hidden], w2 [hidden], b2.
The gradient is pinned in tests/test_mlp_oracle.py by central finite
differences, which share nothing with the chain rule written here.
"""
import numpy as np


def param_count(features: int, hidden: int) -> int:
    return hidden * features + 2 * hidden + 1


def unpack(params, features: int, hidden: int):
    p = np.asarray(params, dtype=np.float64)
    w1 = p[: hidden * features].reshape(hidden, features)
    b1 = p[hidden * features: hidden * features + hidden]
    w2 = p[hidden * features + hidden: hidden * features + 2 * hidden]
    b2 = p[-1]
    return w1, b1, w2, b2


def forward(params, x, features: int, hidden: int) -> np.ndarray:
    w1, b1, w2, b2 = unpack(params, features, hidden)
    pre = np.asarray(x, np.float64) @ w1.T + b1
    return np.maximum(pre, 0.0) @ w2 + b2


def loss(params, x, t, features: int, hidden: int) -> float:
    r = forward(params, x, features, hidden) - np.asarray(t, np.float64)
    return float(np.mean(r * r))


def loss_grad(params, x, t, features: int, hidden: int):
    """(L, dL/dparams) for L = mean((y - t)^2); the ReLU's derivative is taken
    as 0 at a pre-activation of exactly 0."""
    x = np.asarray(x, np.float64)
    t = np.asarray(t, np.float64)
    n = x.shape[0]
    w1, b1, w2, b2 = unpack(params, features, hidden)
    pre = x @ w1.T + b1                 # [n, hidden]
    h = np.maximum(pre, 0.0)
    y = h @ w2 + b2                      # [n]
    r = y - t
    dy = 2.0 * r / n                     # dL/dy
    gw2 = h.T @ dy
    gb2 = dy.sum()
    dpre = np.outer(dy, w2) * (pre > 0)  # dL/dpre
    gw1 = dpre.T @ x
    gb1 = dpre.sum(axis=0)
    grad = np.concatenate([gw1.reshape(-1), gb1, gw2, [gb2]])
    return float(np.mean(r * r)), grad
