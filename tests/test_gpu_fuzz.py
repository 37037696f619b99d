"""Seeded random configurations through the C ABI against the oracle,
bit-exact: single sorts over random key types, sizes (log-uniform, with
ragged tails), bit ranges, key distributions, payloads and pointer offsets;
batches over random segment layouts (empty segments, segments around the
one-block capacity and the tile, long segments) with random bit ranges.
The configurations come from a fixed seed, so every run checks the same
cases."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2206_01784_gb300 import onesweep as osw  # noqa: E402
from paper_2206_01784_gb300 import workload  # noqa: E402

pytestmark = pytest.mark.gpu

KB = {"u32": 32, "u64": 64, "f32": 32, "f64": 64, "i32": 32, "i64": 64}
TYPES = sorted(KB)
DISTS = ["uniform", "and2", "and4", "and8", "const"]


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _to_dev(a, offset=0):
    view = a.view(np.int64 if a.dtype.itemsize == 8 else np.int32)
    dt = torch.int64 if a.dtype.itemsize == 8 else torch.int32
    buf = torch.empty(a.size + offset, dtype=dt, device=_dev())
    buf[offset:] = torch.from_numpy(view.copy()).to(_dev())
    return buf[offset:]


def _keys(kt, dist, n, seed):
    if kt in ("f32", "f64"):
        dist = "normal" if dist == "uniform" else dist
        if dist != "normal":  # the AND bands and all-equal words, read as float bits
            return workload.keys("u64" if KB[kt] == 64 else "u32", dist, n, seed)
    return workload.keys(kt, dist, n, seed)


def _single_cases(count=48, seed=20260):
    rng = np.random.RandomState(seed)
    cases = []
    for i in range(count):
        kt = TYPES[rng.randint(len(TYPES))]
        n = int(np.exp(rng.uniform(0, np.log(400_000))))
        bits = KB[kt]
        if rng.rand() < 0.5:
            begin, end = 0, bits
        else:
            begin = int(rng.randint(0, bits))
            end = int(rng.randint(begin, bits + 1))
        cases.append((i, kt, n, begin, end, DISTS[rng.randint(len(DISTS))], bool(rng.rand() < 0.6),
                      int(rng.randint(0, 4))))
    return cases


@pytest.mark.parametrize("case", _single_cases(), ids=lambda c: f"s{c[0]}-{c[1]}-n{c[2]}-{c[3]}:{c[4]}-{c[5]}")
def test_fuzz_single(case):
    i, kt, n, begin, end, dist, pairs, offset = case
    _dev()
    keys = _keys(kt, dist, n, seed=1000 + i)
    vals = workload.iota_u32(n) if pairs else None
    k = _to_dev(keys, offset)
    dt = np.uint64 if KB[kt] == 64 else np.uint32
    if pairs:
        ko, vo = osw.sort_pairs(k, _to_dev(vals, offset), begin, end, key_type=kt)
        torch.cuda.synchronize()
        exp = oracle.sort(kt, keys, vals, begin, end)
        assert np.array_equal(ko.cpu().numpy().view(dt), exp[0])
        assert np.array_equal(vo.cpu().numpy().view(np.uint32), exp[1])
    else:
        ko = osw.sort_keys(k, begin, end, key_type=kt)
        torch.cuda.synchronize()
        assert np.array_equal(ko.cpu().numpy().view(dt), oracle.sort(kt, keys, None, begin, end))


def _batch_cases(count=16, seed=20261):
    rng = np.random.RandomState(seed)
    cases = []
    for i in range(count):
        kt = TYPES[rng.randint(len(TYPES))]
        segs = int(rng.randint(1, 300))
        kind = rng.rand(segs)
        sizes = np.where(kind < 0.15, 0,
                         np.where(kind < 0.6, rng.randint(1, 5000, segs),
                                  np.where(kind < 0.9, rng.randint(5000, 20000, segs), rng.randint(20000, 150000, segs))))
        bits = KB[kt]
        begin, end = (0, bits) if rng.rand() < 0.6 else (int(rng.randint(0, bits // 2)), bits)
        cases.append((i, kt, sizes.astype(np.int64), begin, end, bool(rng.rand() < 0.6)))
    return cases


@pytest.mark.parametrize("case", _batch_cases(), ids=lambda c: f"b{c[0]}-{c[1]}-segs{len(c[2])}")
def test_fuzz_batch(case):
    i, kt, sizes, begin, end, pairs = case
    _dev()
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offs[-1])
    keys = _keys(kt, "and2" if i % 2 else "uniform", n, seed=2000 + i)
    vals = workload.iota_u32(n) if pairs else None
    o = torch.from_numpy(offs).to(_dev())
    dt = np.uint64 if KB[kt] == 64 else np.uint32
    exp = oracle.sort_segments(kt, keys, offs.astype(np.uint64), vals, begin, end)
    if pairs:
        ko, vo = osw.sort_batch(_to_dev(keys), o, _to_dev(vals), begin, end, key_type=kt)
        torch.cuda.synchronize()
        assert np.array_equal(ko.cpu().numpy().view(dt), exp[0])
        assert np.array_equal(vo.cpu().numpy().view(np.uint32), exp[1])
    else:
        ko = osw.sort_batch(_to_dev(keys), o, None, begin, end, key_type=kt)
        torch.cuda.synchronize()
        assert np.array_equal(ko.cpu().numpy().view(dt), exp)
