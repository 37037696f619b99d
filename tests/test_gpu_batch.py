"""Segmented (batched) sort through the C ABI against the oracle, bit-exact.

Each segment is sorted on its own (``oracle.sort_segments``). Covers empty and
one-key segments, segments at and around the one-block capacity and the
binning tile, many-tile segments, all key types, keys only and pairs, bit
ranges, invalid offsets, CUDA-graph capture, and equality with one
os_sort_pairs call per segment.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2206_01784_gb300 import onesweep as osw  # noqa: E402
from paper_2206_01784_gb300 import workload  # noqa: E402

pytestmark = pytest.mark.gpu

KB = {"u32": 32, "u64": 64, "f32": 32, "f64": 64, "i32": 32, "i64": 64}


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev(a):
    return torch.from_numpy(a.view(np.int64 if a.dtype.itemsize == 8 else np.int32).copy()).to(_dev())


def kdtype(kt):
    return np.uint64 if KB[kt] == 64 else np.uint32


def make_keys(kt, n, seed, dist="and2"):
    if kt in ("f32", "f64"):
        return workload.keys(kt, "normal", n, seed)
    return workload.keys(kt, dist, n, seed)


def run_batch(kt, keys, sizes, pairs, begin=0, end=None):
    end = KB[kt] if end is None else end
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offs[-1])
    vals = workload.iota_u32(n) if pairs else None
    k = to_dev(keys)
    o = torch.from_numpy(offs).to(_dev())
    if pairs:
        ko, vo = osw.sort_batch(k, o, to_dev(vals), begin, end, key_type=kt)
        torch.cuda.synchronize()
        got = (ko.cpu().numpy().view(kdtype(kt)), vo.cpu().numpy().view(np.uint32))
    else:
        ko = osw.sort_batch(k, o, None, begin, end, key_type=kt)
        torch.cuda.synchronize()
        got = ko.cpu().numpy().view(kdtype(kt))
    exp = oracle.sort_segments(kt, keys, offs.astype(np.uint64), vals, begin, end)
    return got, exp


def edge_sizes(kt, pairs):
    cap = 4096 if KB[kt] == 32 else 2048  # one-block capacity
    cfg = osw.os_get_tile_config(KB[kt], 4 if pairs else 0)
    if cfg % 4 == 3:  # the persistent geometry serves single arrays; a batch runs geometry 0
        cfg -= 3
    t = osw.os_tile_config_keys(KB[kt], 4 if pairs else 0, cfg)
    return [0, 1, 2, 31, 33, cap - 1, cap, cap + 1, 0, t - 1, t, t + 1, 3 * t + 7, 1000, 0, 5, 2 * cap + 3]


@pytest.mark.parametrize("kt", ["u32", "u64", "f32", "f64", "i32", "i64"])
@pytest.mark.parametrize("pairs", [False, True])
def test_batch_edge_segments(kt, pairs):
    sizes = edge_sizes(kt, pairs)
    keys = make_keys(kt, sum(sizes), seed=3)
    got, exp = run_batch(kt, keys, sizes, pairs)
    if pairs:
        assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])
    else:
        assert np.array_equal(got, exp)


@pytest.mark.parametrize("dist", ["uniform", "and3", "and8", "const"])
def test_batch_lognormal_segments(dist):
    sizes = workload.segment_sizes(300, seed=10, median=6000.0, sigma=1.18, lo=64, hi=200_000)
    keys = make_keys("u32", int(sizes.sum()), seed=11, dist=dist)
    got, exp = run_batch("u32", keys, sizes, True)
    assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])


@pytest.mark.parametrize("begin,end", [(0, 8), (3, 29), (16, 32), (5, 5)])
def test_batch_bit_ranges(begin, end):
    sizes = [100, 9000, 0, 4096, 25000, 3]
    keys = make_keys("u32", sum(sizes), seed=12, dist="uniform")
    got, exp = run_batch("u32", keys, sizes, True, begin, end)
    assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])


def test_batch_one_segment_equals_single_sort():
    n = 700_001
    keys = make_keys("u32", n, seed=13, dist="uniform")
    got, _ = run_batch("u32", keys, [n], True)
    exp = oracle.sort("u32", keys, workload.iota_u32(n))
    assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])


def test_batch_matches_per_array_calls():
    sizes = workload.segment_sizes(64, seed=14, median=20000.0, sigma=1.18, lo=1024, hi=300_000)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offs[-1])
    keys = make_keys("u32", n, seed=15, dist="uniform")
    k, v = to_dev(keys), to_dev(workload.iota_u32(n))
    bk, bv = osw.sort_batch(k, torch.from_numpy(offs).to(_dev()), v, key_type="u32")
    pk, pv = torch.empty_like(k), torch.empty_like(v)
    for s in range(len(sizes)):
        lo, hi = int(offs[s]), int(offs[s + 1])
        osw.sort_pairs(k[lo:hi], v[lo:hi], key_type="u32", keys_out=pk[lo:hi], values_out=pv[lo:hi])
    torch.cuda.synchronize()
    assert torch.equal(bk, pk) and torch.equal(bv, pv)


def test_batch_invalid_offsets_reported():
    n = 10_000
    keys = make_keys("u32", n, seed=16)
    k = to_dev(keys)
    out = torch.empty_like(k)
    for bad in ([0, 5000, 4000, n], [0, 3000, n + 5]):
        offs = torch.tensor(bad, dtype=torch.int64, device=_dev())
        segs = len(bad) - 1
        ws = osw.batch_workspace(osw.OS_KEY_U32, n, segs, 0, 0, 32, k.device)
        s = torch.cuda.current_stream().cuda_stream
        rc = osw.os_sort_batch(osw.OS_KEY_U32, k.data_ptr(), out.data_ptr(), None, None, offs.data_ptr(), segs, n, 0,
                               32, ws.data_ptr(), ws.numel(), s)
        assert rc == osw.OS_OK
        assert osw.os_workspace_status(ws.data_ptr(), s) == osw.OS_ERR_INVALID_ARG


def test_batch_cuda_graph_replay():
    # one capture, replayed on new data with new segment boundaries of the
    # same count and total
    dev = _dev()
    n, segs = 200_000, 37
    k = torch.empty(n, dtype=torch.int32, device=dev)
    v = torch.empty(n, dtype=torch.int32, device=dev)
    offs = torch.empty(segs + 1, dtype=torch.int64, device=dev)
    ko, vo = torch.empty_like(k), torch.empty_like(v)
    ws = osw.batch_workspace(osw.OS_KEY_U32, n, segs, 4, 0, 32, dev)

    def fill(seed):
        rng = np.random.default_rng(seed)
        cuts = np.sort(rng.integers(0, n, segs - 1))
        o = np.concatenate([[0], cuts, [n]]).astype(np.int64)
        keys = make_keys("u32", n, seed=seed, dist="uniform")
        k.copy_(torch.from_numpy(keys.view(np.int32)))
        v.copy_(torch.from_numpy(workload.iota_u32(n).view(np.int32)))
        offs.copy_(torch.from_numpy(o))
        return keys, o

    fill(1)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        osw.sort_batch(k, offs, v, key_type="u32", keys_out=ko, values_out=vo, ws=ws, stream=s)  # warm-up
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        osw.sort_batch(k, offs, v, key_type="u32", keys_out=ko, values_out=vo, ws=ws)
    for seed in (2, 3):
        keys, o = fill(seed)
        g.replay()
        torch.cuda.synchronize()
        ek, ev = oracle.sort_segments("u32", keys, o.astype(np.uint64), workload.iota_u32(n))
        assert np.array_equal(ko.cpu().numpy().view(np.uint32), ek)
        assert np.array_equal(vo.cpu().numpy().view(np.uint32), ev)


@pytest.mark.parametrize("cfg", list(range(12)))
def test_batch_every_tile_config(cfg):
    # a batch with the persistent variant selected runs geometry 0 (same ranking)
    prev = osw.os_get_tile_config(32, 4)
    try:
        assert osw.os_set_tile_config(32, 4, cfg) == osw.OS_OK
        sizes = edge_sizes("u32", True) + [50_000]
        keys = make_keys("u32", sum(sizes), seed=20 + cfg)
        got, exp = run_batch("u32", keys, sizes, True)
        assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])
    finally:
        osw.os_set_tile_config(32, 4, prev)
