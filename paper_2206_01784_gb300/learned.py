"""Learned cost model for scheduling sorts (not part of the sorting method).

A one-hidden-layer ReLU perceptron maps a sort's features - log2 of its key
count, its key width and type, whether it carries values - to the log of its
device time. Training data are times measured on this GPU: ``collect`` times
whole sorts, ``collect_batched`` a request's share of a batched sort (what
the coalescing service pays per request). Training runs on the GPU with the
library's own kernels (os_mlp_loss_grad, os_mlp_adam_step in
include/onesweep_mlp.h). The sort service uses the predictions to admit
waiting requests shortest-predicted-first instead of first-come-first-served
(``serve.Admission(order=...)``), evaluating the trained network on the host
from a parameter copy (``priority``). The network never sees keys: every
sort's output is the same whatever it predicts.
"""
from __future__ import annotations

import math

import numpy as np

from . import onesweep as osw
from . import workload

FEATURES = ("log2_keys", "u64", "f32", "pairs")
KEY_TYPES = ("u32", "u64", "f32")


def features(key_type: str, n: int, pairs: bool = True) -> list[float]:
    return [math.log2(max(n, 1)) / 16.0, 1.0 if key_type in ("u64", "f64") else 0.0,
            1.0 if key_type in ("f32", "f64") else 0.0, 1.0 if pairs else 0.0]


def collect(sizes_log2=range(10, 25), key_types=KEY_TYPES, reps: int = 3, seed: int = 3):
    """Measured (features, log ms) of single sorts of u32-valued pairs on the
    current GPU (CUDA events around each os_sort_pairs call)."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    s = torch.cuda.current_stream(dev)
    X, T = [], []
    for kt in key_types:
        kb = 64 if kt in ("u64", "f64") else 32
        for lg in sizes_log2:
            n = 1 << lg
            keys = workload.keys(kt if kt != "f32" else "f32", "normal" if kt == "f32" else "uniform", n, seed + lg)
            k = torch.from_numpy(keys.view(np.int64 if kb == 64 else np.int32)).to(dev)
            v = torch.from_numpy(workload.iota_u32(n).view(np.int32)).to(dev)
            ko, vo = torch.empty_like(k), torch.empty_like(v)
            ws = osw.workspace(osw.KEY_TYPES[kt], n, 4, 0, kb, dev)
            for r in range(reps + 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                rc = osw.os_sort_pairs(osw.KEY_TYPES[kt], k.data_ptr(), ko.data_ptr(), v.data_ptr(), vo.data_ptr(),
                                       n, 0, kb, ws.data_ptr(), ws.numel(), s.cuda_stream)
                e1.record(s)
                if rc != osw.OS_OK:
                    raise osw.OnesweepError(rc, "os_sort_pairs")
                e1.synchronize()
                if r > 0:  # the first call warms up
                    X.append(features(kt, n))
                    T.append(math.log(e0.elapsed_time(e1)))
    return np.array(X, np.float32), np.array(T, np.float32)


def collect_batched(sizes_log2=range(10, 23, 2), key_types=KEY_TYPES, batch_keys: int = 1 << 22, reps: int = 3,
                    seed: int = 5):
    """Measured (features, log ms) of a request's share of a batch: for each
    key type and size n, the device time of one os_sort_batch of k equal
    segments of n keys (k * n near batch_keys, 4 <= k <= 1024) divided by k.
    This is what a request costs the sort service, which coalesces requests
    into batches: per-launch costs are shared, the per-key work of the key
    type is not."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    s = torch.cuda.current_stream(dev)
    X, T = [], []
    for kt in key_types:
        kb = 64 if kt in ("u64", "f64") else 32
        for lg in sizes_log2:
            n = 1 << lg
            k = max(4, min(1024, batch_keys // n))
            keys = workload.keys(kt, "normal" if kt == "f32" else "uniform", n * k, seed + lg)
            kd = torch.from_numpy(keys.view(np.int64 if kb == 64 else np.int32)).to(dev)
            vd = torch.from_numpy(workload.iota_u32(n * k).view(np.int32)).to(dev)
            offs = torch.arange(0, (k + 1) * n, n, dtype=torch.int64, device=dev)
            ws = osw.batch_workspace(osw.KEY_TYPES[kt], n * k, k, 4, 0, kb, dev)
            ko, vo = torch.empty_like(kd), torch.empty_like(vd)
            times = []
            for r in range(reps + 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                osw.sort_batch(kd, offs, values=vd, key_type=kt, keys_out=ko, values_out=vo, ws=ws)
                e1.record(s)
                e1.synchronize()
                if r > 0:  # the first call warms up
                    times.append(e0.elapsed_time(e1) / k)
            X.append(features(kt, n))
            T.append(math.log(float(np.median(times))))
            del kd, vd, ko, vo, ws
    return np.array(X, np.float32), np.array(T, np.float32)


class CostModel:
    """The perceptron, its parameters and Adam state on the GPU."""

    def __init__(self, hidden: int = 32, seed: int = 0, device=None):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.f, self.h = len(FEATURES), hidden
        count = osw.os_mlp_param_count(self.f, self.h)
        rng = np.random.default_rng(seed)
        p = np.zeros(count, np.float32)
        p[: self.h * self.f] = rng.normal(scale=math.sqrt(2.0 / self.f), size=self.h * self.f)
        p[self.h * self.f: self.h * self.f + self.h] = 0.1
        p[self.h * self.f + self.h: self.h * self.f + 2 * self.h] = rng.normal(scale=math.sqrt(1.0 / self.h),
                                                                                size=self.h)
        self.params = torch.from_numpy(p).to(self.device)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.step = 0
        self._host = None  # (W1, b1, w2, b2) in host memory, taken after training

    def _stream(self):
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def loss_grad(self, x, t):
        """(loss, gradient) on device tensors x [n, f], t [n] (float32)."""
        n = x.shape[0]
        rc = osw.os_mlp_loss_grad(self.params.data_ptr(), self.f, self.h, x.data_ptr(), t.data_ptr(), n,
                                  self.grads.data_ptr(), self.loss.data_ptr(), self._stream())
        if rc != osw.OS_OK:
            raise osw.OnesweepError(rc, "os_mlp_loss_grad")
        return self.loss, self.grads

    def fit(self, X: np.ndarray, T: np.ndarray, steps: int = 3000, lr: float = 3e-3, log_every: int = 500):
        torch = self.torch
        x = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(self.device)
        t = torch.from_numpy(np.ascontiguousarray(T, np.float32)).to(self.device)
        history = []
        for i in range(steps):
            self.loss_grad(x, t)
            self.step += 1
            rc = osw.os_mlp_adam_step(self.params.data_ptr(), self.grads.data_ptr(), self.m.data_ptr(),
                                      self.v.data_ptr(), self.params.numel(), lr, 0.9, 0.999, 1e-8, self.step,
                                      self._stream())
            if rc != osw.OS_OK:
                raise osw.OnesweepError(rc, "os_mlp_adam_step")
            if i % log_every == 0 or i == steps - 1:
                history.append(float(self.loss.item()))
        self.host_copy()
        return history

    def host_copy(self):
        """The trained parameters copied to host memory once: (W1 [hidden,
        features], b1 [hidden], w2 [hidden], b2), the layout of
        include/onesweep_mlp.h."""
        p = self.params.cpu().numpy().astype(np.float32)
        f, h = self.f, self.h
        self._host = (p[: h * f].reshape(h, f), p[h * f: h * f + h], p[h * f + h: h * f + 2 * h], p[h * f + 2 * h])
        return self._host

    def predict_log_ms_host(self, X: np.ndarray) -> np.ndarray:
        """The same network evaluated on the host from the copy of its
        parameters (float32): pre = W1 x + b1, y = w2 . max(pre, 0) + b2."""
        w1, b1, w2, b2 = self._host if self._host is not None else self.host_copy()
        x = np.ascontiguousarray(X, np.float32)
        return np.maximum(x @ w1.T + b1, 0.0) @ w2 + b2

    def predict_log_ms(self, X: np.ndarray) -> np.ndarray:
        torch = self.torch
        x = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(self.device)
        y = torch.empty(x.shape[0], dtype=torch.float32, device=self.device)
        rc = osw.os_mlp_forward(self.params.data_ptr(), self.f, self.h, x.data_ptr(), x.shape[0], y.data_ptr(),
                                self._stream())
        if rc != osw.OS_OK:
            raise osw.OnesweepError(rc, "os_mlp_forward")
        return y.cpu().numpy()

    def priority(self, requests) -> dict:
        """Predicted device ms of each request (id -> ms), for shortest-first
        admission. Evaluated on the host from the parameters copied after
        training: the service calls this every tick, and a device call there
        would wait for every sort in flight (a copy back to the host on the
        default stream synchronizes with the service's streams), which
        measured on GB300 doubled the mean latency of a burst."""
        X = np.array([features(r.key_type, r.n) for r in requests], np.float32)
        ms = np.exp(self.predict_log_ms_host(X)) if len(requests) else np.zeros(0)
        return {id(r): float(v) for r, v in zip(requests, ms)}
