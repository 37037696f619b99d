"""Sort of one array across ranks (MSD split, one all-to-all), on CPU with gloo.

The exchange logic is the package's own (sharded.py); the local steps (top
place histogram, stable partition, local sort) run through a backend, which
here is the CPU oracle, so the test checks the split and the exchange against
the oracle's sort of the whole array, element by element (index values make
stability visible).
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

# ------------------------------------------------------------------ planning


def test_top_place():
    assert sharded.top_place(0, 32) == (24, 32)
    assert sharded.top_place(0, 64) == (56, 64)
    assert sharded.top_place(4, 30) == (28, 30)   # places 4,12,20,28: the top one 2 bits wide
    assert sharded.top_place(3, 11) == (3, 11)
    assert sharded.top_place(5, 5) == (5, 5)


def _check_bounds(hist, world, bounds):
    assert len(bounds) == world + 1 and bounds[0] == 0 and bounds[-1] == len(hist)
    assert all(a <= b for a, b in zip(bounds, bounds[1:]))
    total = sum(hist)
    biggest = max(hist) if hist else 0
    cum = np.concatenate([[0], np.cumsum(hist)])
    for j in range(1, world):
        # every inner boundary is within one bin of its ideal cut
        assert abs(cum[bounds[j]] - j * total / world) <= biggest


def test_plan_split_uniform():
    hist = [10] * 256
    b = sharded.plan_split(hist, 4)
    assert b == [0, 64, 128, 192, 256]
    _check_bounds(hist, 4, b)


def test_plan_split_one_bin():
    hist = [0] * 256
    hist[77] = 1000
    for world in (2, 3, 8):
        b = sharded.plan_split(hist, world)
        _check_bounds(hist, world, b)
        loads = sharded.send_counts(hist, b)
        assert sorted(loads)[-1] == 1000 and sum(loads) == 1000


def test_plan_split_random():
    rng = np.random.default_rng(0)
    for trial in range(200):
        nb = int(rng.integers(1, 300))
        world = int(rng.integers(1, 12))
        hist = [int(x) for x in rng.integers(0, 50, nb) * (rng.random(nb) < 0.7)]
        b = sharded.plan_split(hist, world)
        _check_bounds(hist, world, b)
        assert sum(sharded.send_counts(hist, b)) == sum(hist)
        assert sharded.plan_split(hist, world) == b          # deterministic


def test_plan_split_empty_and_world_one():
    b = sharded.plan_split([0] * 256, 3)
    _check_bounds([0] * 256, 3, b)
    assert sharded.send_counts([0] * 256, b) == [0, 0, 0]
    assert sharded.plan_split([5] * 16, 1) == [0, 16]
    with pytest.raises(ValueError):
        sharded.plan_split([1], 0)


def test_send_counts():
    assert sharded.send_counts([1, 2, 3, 4], [0, 1, 3, 4]) == [1, 5, 4]

# ------------------------------------------------------------- exchange (gloo)


class OracleBackend:
    """The local steps on the CPU oracle (test infrastructure only)."""

    def __init__(self, key_type, descending=False):
        self.kt = key_type
        self.desc = descending

    def _np(self, t):
        return t.numpy().view(oracle._key_dtype(self.kt))

    def top_histogram(self, keys, lo, hi):
        h = oracle.histograms(self.kt, self._np(keys), lo, hi, descending=self.desc)
        return [int(x) for x in h[0][:1 << (hi - lo)]]

    def partition(self, keys, values, lo, hi):
        return self.sort(keys, values, lo, hi)

    def sort(self, keys, values, begin, end):
        k = self._np(keys)
        if values is None:
            ok = oracle.sort(self.kt, k, begin_bit=begin, end_bit=end, descending=self.desc)
            return torch.from_numpy(ok.view(keys.numpy().dtype).copy()), None
        ok, ov = oracle.sort(self.kt, k, values.numpy().view(np.uint32), begin_bit=begin, end_bit=end,
                             descending=self.desc)
        return torch.from_numpy(ok.view(keys.numpy().dtype).copy()), torch.from_numpy(ov.view(np.int32).copy())


_INT = {"u32": np.int32, "i32": np.int32, "f32": np.int32, "u64": np.int64, "i64": np.int64, "f64": np.int64}

CASES = [
    # key type, distribution, n, pieces (fractions), pairs, begin, end, descending
    ("u32", "uniform", 60001, (0.4, 0.6), True, 0, 32, False),
    ("u32", "and3", 50000, (0.5, 0.5), True, 0, 32, False),
    ("u32", "const", 20000, (0.3, 0.7), True, 0, 32, False),
    ("f32", "normal", 40000, (0.5, 0.5), True, 0, 32, True),
    ("i64", "uniform", 30000, (0.7, 0.3), False, 4, 60, False),
    ("u32", "uniform", 25000, (0.0, 1.0), True, 0, 32, False),   # rank 0 holds nothing
    ("u64", "and2", 30000, (0.2, 0.3, 0.5), True, 0, 64, False),
    ("i32", "uniform", 30000, (0.5, 0.25, 0.25), True, 0, 32, True),
]


def _case_input(case):
    kt, distn, n, _, _, _, _, _ = case
    keys = workload.keys(kt, distn, n, seed=n % 97)
    return keys, workload.iota_u32(n)


def _pieces(n, fracs):
    cuts = [0]
    for f in fracs[:-1]:
        cuts.append(cuts[-1] + int(round(f * n)))
    cuts.append(n)
    return cuts


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = {}
        for ci, case in enumerate(CASES):
            kt, _, n, fracs, pairs, begin, end, desc = case
            if len(fracs) != world:
                continue
            keys, vals = _case_input(case)
            cuts = _pieces(n, fracs)
            lo, hi = cuts[rank], cuts[rank + 1]
            k = torch.from_numpy(keys[lo:hi].view(_INT[kt]).copy())
            v = torch.from_numpy(vals[lo:hi].view(np.int32).copy()) if pairs else None
            ok, ov, plan = sharded.sharded_sort(k, v, begin, end, backend=OracleBackend(kt, desc))
            out[ci] = (ok.numpy().tobytes(), None if ov is None else ov.numpy().tobytes(), plan.bounds,
                       plan.send, plan.recv)
        dist.barrier()
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def _run(world):
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_sort_matches_oracle(world):
    res = _run(world)
    checked = 0
    for ci, case in enumerate(CASES):
        kt, distn, n, fracs, pairs, begin, end, desc = case
        if len(fracs) != world:
            continue
        keys, vals = _case_input(case)
        dt = oracle._key_dtype(kt)
        got_k = np.concatenate([np.frombuffer(res[r][ci][0], dtype=dt) for r in range(world)])
        if pairs:
            ek, ev = oracle.sort(kt, keys, vals, begin_bit=begin, end_bit=end, descending=desc)
            got_v = np.concatenate([np.frombuffer(res[r][ci][1], dtype=np.uint32) for r in range(world)])
            assert np.array_equal(got_v, ev), case
        else:
            ek = oracle.sort(kt, keys, begin_bit=begin, end_bit=end, descending=desc)
        assert np.array_equal(got_k, ek), case
        # every rank agreed on the split, and what was sent is what was received
        bounds = [res[r][ci][2] for r in range(world)]
        assert all(b == bounds[0] for b in bounds)
        send = np.array([res[r][ci][3] for r in range(world)])
        recv = np.array([res[r][ci][4] for r in range(world)])
        assert np.array_equal(send.T, recv)
        assert send.sum() == n
        checked += 1
    assert checked > 0
