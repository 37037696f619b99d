"""Pins of the cost model's reference gradient (no GPU): central finite
differences in float64, and the linear special case's closed form."""
import numpy as np

from oracle import mlp_oracle as mo


def _problem(seed, f=5, h=7, n=40):
    rng = np.random.default_rng(seed)
    params = rng.normal(size=mo.param_count(f, h)) * 0.5
    x = rng.normal(size=(n, f))
    t = rng.normal(size=n)
    return params, x, t, f, h


def test_gradient_matches_finite_differences():
    for seed in range(3):
        params, x, t, f, h = _problem(seed)
        _, g = mo.loss_grad(params, x, t, f, h)
        eps = 1e-6
        num = np.empty_like(params)
        for i in range(params.size):
            p1, p2 = params.copy(), params.copy()
            p1[i] += eps
            p2[i] -= eps
            num[i] = (mo.loss(p1, x, t, f, h) - mo.loss(p2, x, t, f, h)) / (2 * eps)
        assert np.allclose(g, num, rtol=1e-5, atol=1e-8)


def test_linear_special_case():
    # one hidden unit that is always active: y = w2 (W1 x + b1) + b2 is linear,
    # so dL/db2 = mean(2 r) and dL/dw2 = mean(2 r * pre)
    f, h = 3, 1
    rng = np.random.default_rng(7)
    x = rng.uniform(1, 2, size=(30, f))
    params = np.array([0.3, 0.2, 0.1, 5.0, 0.7, -0.4])  # W1, b1 (keeps pre > 0), w2, b2
    t = rng.normal(size=30)
    pre = x @ params[:3] + params[3]
    y = 0.7 * pre - 0.4
    r = y - t
    L, g = mo.loss_grad(params, x, t, f, h)
    assert abs(L - np.mean(r * r)) < 1e-12
    assert abs(g[-1] - np.mean(2 * r)) < 1e-12
    assert abs(g[-2] - np.mean(2 * r * pre)) < 1e-12
    assert np.allclose(g[:3], (2 * r * 0.7) @ x / 30)
