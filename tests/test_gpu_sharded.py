"""Sort of one array across ranks with the CUDA backend, against the oracle.

Two ranks run as two processes on the one GPU this suite gets, exchanging
through gloo (host memory); every local step (top-place histogram, stable
partition, local sort) runs the library's kernels. The kernels of the two
processes never wait on each other: the only rendezvous is gloo's, on the
host, between launches.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2206_01784_gb300 import sharded, workload

pytestmark = pytest.mark.gpu

_INT = {"u32": np.int32, "i32": np.int32, "f32": np.int32, "u64": np.int64, "i64": np.int64, "f64": np.int64}

CASES = [
    # key type, distribution, n, piece of rank 0, pairs, begin, end, descending
    ("u32", "uniform", (1 << 22) + 5, 0.45, True, 0, 32, False),
    ("u32", "and3", 1 << 21, 0.5, True, 0, 32, False),
    ("f32", "normal", (1 << 21) + 3, 0.6, True, 0, 32, True),
    ("u64", "uniform", 1 << 20, 0.5, False, 0, 64, False),
    ("i32", "uniform", 300001, 0.0, True, 3, 29, False),
    ("u32", "const", 1 << 20, 0.5, True, 0, 32, False),
]


def _input(case):
    kt, distn, n = case[:3]
    return workload.keys(kt, distn, n, seed=(n % 89) + 1), workload.iota_u32(n)


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = {}
        for ci, case in enumerate(CASES):
            kt, _, n, frac, pairs, begin, end, desc = case
            keys, vals = _input(case)
            cut = int(round(frac * n))
            lo, hi = (0, cut) if rank == 0 else (cut, n)
            dev = torch.device("cuda:0")
            k = torch.from_numpy(keys[lo:hi].view(_INT[kt]).copy()).to(dev)
            v = torch.from_numpy(vals[lo:hi].view(np.int32).copy()).to(dev) if pairs else None
            ok, ov, plan = sharded.sharded_sort(k, v, begin, end, backend=sharded.CudaBackend(kt, desc))
            torch.cuda.synchronize()
            out[ci] = (ok.cpu().numpy().tobytes(), None if ov is None else ov.cpu().numpy().tobytes(), plan.bounds)
        dist.barrier()
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_ranks_on_cuda_backend():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for ci, case in enumerate(CASES):
        kt, _, n, frac, pairs, begin, end, desc = case
        keys, vals = _input(case)
        dt = oracle._key_dtype(kt)
        got_k = np.concatenate([np.frombuffer(res[r][ci][0], dtype=dt) for r in range(2)])
        if pairs:
            ek, ev = oracle.sort(kt, keys, vals, begin_bit=begin, end_bit=end, descending=desc)
            got_v = np.concatenate([np.frombuffer(res[r][ci][1], dtype=np.uint32) for r in range(2)])
            assert np.array_equal(got_v, ev), case
        else:
            ek = oracle.sort(kt, keys, begin_bit=begin, end_bit=end, descending=desc)
        assert np.array_equal(got_k, ek), case
        assert res[0][ci][2] == res[1][ci][2]
