"""The cost model's CUDA kernels against the float64 oracle, its training on
measured sort times, and what it gains the sort service: shortest-predicted-
first admission against first-come-first-served on the same burst."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp_oracle as mo  # noqa: E402
from paper_2206_01784_gb300 import learned  # noqa: E402
from paper_2206_01784_gb300 import onesweep as osw  # noqa: E402
from paper_2206_01784_gb300 import serve  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("f,h,n", [(4, 32, 1000), (7, 13, 257), (32, 128, 64), (1, 1, 3)])
def test_forward_and_gradient_match_oracle(f, h, n):
    dev = _dev()
    rng = np.random.default_rng(f * 100 + h)
    p = (rng.normal(size=mo.param_count(f, h)) * 0.3).astype(np.float32)
    x = rng.normal(size=(n, f)).astype(np.float32)
    t = rng.normal(size=n).astype(np.float32)
    pd, xd, td = (torch.from_numpy(a).to(dev) for a in (p, x, t))
    y = torch.empty(n, dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream().cuda_stream
    assert osw.os_mlp_forward(pd.data_ptr(), f, h, xd.data_ptr(), n, y.data_ptr(), s) == osw.OS_OK
    g = torch.empty_like(pd)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    assert osw.os_mlp_loss_grad(pd.data_ptr(), f, h, xd.data_ptr(), td.data_ptr(), n, g.data_ptr(),
                                loss.data_ptr(), s) == osw.OS_OK
    torch.cuda.synchronize()
    ref_y = mo.forward(p.astype(np.float64), x.astype(np.float64), f, h)
    ref_l, ref_g = mo.loss_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), f, h)
    # float32 arithmetic (and atomic summation order) against float64
    assert np.allclose(y.cpu().numpy(), ref_y, rtol=1e-4, atol=1e-4)
    assert abs(loss.item() - ref_l) <= 1e-4 * max(1.0, ref_l)
    scale = np.abs(ref_g).max()
    assert np.allclose(g.cpu().numpy(), ref_g, rtol=1e-3, atol=1e-4 * scale)


def test_adam_step_matches_formula():
    dev = _dev()
    rng = np.random.default_rng(1)
    p, g = rng.normal(size=50).astype(np.float32), rng.normal(size=50).astype(np.float32)
    m, v = np.zeros(50, np.float32), np.zeros(50, np.float32)
    pd, gd, md, vd = (torch.from_numpy(a.copy()).to(dev) for a in (p, g, m, v))
    s = torch.cuda.current_stream().cuda_stream
    for step in (1, 2):
        assert osw.os_mlp_adam_step(pd.data_ptr(), gd.data_ptr(), md.data_ptr(), vd.data_ptr(), 50, 0.01, 0.9, 0.999,
                                    1e-8, step, s) == osw.OS_OK
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        p = p - 0.01 * (m / (1 - 0.9 ** step)) / (np.sqrt(v / (1 - 0.999 ** step)) + 1e-8)
    assert np.allclose(pd.cpu().numpy(), p, rtol=1e-5, atol=1e-6)


def test_training_fits_measured_sort_times():
    _dev()
    X, T = learned.collect(sizes_log2=range(10, 23, 2), reps=2)
    model = learned.CostModel(hidden=32, seed=0)
    hist = model.fit(X, T, steps=2500, lr=3e-3)
    assert hist[-1] < 0.1 * hist[0]
    pred = model.predict_log_ms(X)
    # within 30 % on the log scale's back-transform for the training points
    assert np.median(np.abs(np.exp(pred - T) - 1.0)) < 0.3


def test_batched_costs_fit_and_host_predictions_match_the_kernel():
    _dev()
    X, T = learned.collect_batched(sizes_log2=range(10, 23, 2), reps=2)
    # a request's share of a batch grows with its keys, and 64-bit keys cost more
    t = np.exp(T).reshape(3, -1)
    assert np.all(np.diff(t[:, 2:], axis=1) > 0)
    assert np.all(t[1, 3:] > 1.5 * t[0, 3:])
    model = learned.CostModel(hidden=32, seed=0)
    hist = model.fit(X, T, steps=2500, lr=3e-3)
    assert hist[-1] < 0.05 * hist[0]
    # the service evaluates the network on the host from a parameter copy:
    # the same function as the forward kernel, to float32 rounding
    assert np.allclose(model.predict_log_ms_host(X), model.predict_log_ms(X), atol=1e-4)


def test_shortest_predicted_first_beats_fifo_on_a_burst():
    _dev()
    X, T = learned.collect_batched(sizes_log2=range(10, 23, 2), reps=2)
    model = learned.CostModel(hidden=32, seed=0)
    model.fit(X, T, steps=2500, lr=3e-3)
    # a 256 MB budget and 1M-key batches serialise the burst, so the order of
    # admission decides how long small requests wait
    srv = serve.Server(budget_bytes=256 << 20, pool_words=1 << 24)

    def burst():
        reqs = serve.make_requests(200, seed=9, rate_per_s=1.0, lo_log2=10, hi_log2=22)
        for r in reqs:
            r.arrival = 0.0
        return reqs

    srv.run(burst(), realtime=False, max_batch_keys=1 << 20)  # warm-up: first launches load kernels
    runs = {"fifo": [], "sjf": []}
    for _ in range(2):
        runs["fifo"].append(srv.run(burst(), realtime=False, max_batch_keys=1 << 20))
        runs["sjf"].append(srv.run(burst(), realtime=False, max_batch_keys=1 << 20, order=model.priority))
    fifo = min(runs["fifo"], key=lambda r: r["mean_ms"])
    sjf = min(runs["sjf"], key=lambda r: r["mean_ms"])
    print(f"burst: fifo mean {fifo['mean_ms']:.2f} p50 {fifo['p50_ms']:.2f}; "
          f"predicted-shortest-first mean {sjf['mean_ms']:.2f} p50 {sjf['p50_ms']:.2f} ms")
    # the same work, but small requests no longer wait behind large ones
    assert sjf["keys"] == fifo["keys"]
    assert sjf["mean_ms"] < 0.85 * fifo["mean_ms"], (sjf["mean_ms"], fifo["mean_ms"])
    assert sjf["p50_ms"] < 0.6 * fifo["p50_ms"], (sjf["p50_ms"], fifo["p50_ms"])
