"""Stable descending order (OS_SORT_DESCENDING OR'd into the key type)
through the C ABI, bit-exact against the CPU oracle's descending sort: every
key type, keys only and pairs, several tiles with ragged tails, narrow and
odd bit ranges, skewed and all-equal keys, every binning variant, the
segmented batch sort and its one-block path, and the histograms and offsets
a descending sort bins by."""
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


def _to_dev(a):
    return torch.from_numpy(a.view(np.int64 if a.dtype.itemsize == 8 else np.int32).copy()).to(_dev())


def _kd(kt):
    return np.uint64 if KB[kt] == 64 else np.uint32


def _keys(kt, dist, n, seed):
    if kt in ("f32", "f64") and dist == "uniform":
        dist = "normal"
    return workload.keys(kt, dist, n, seed)


@pytest.mark.parametrize("kt", ["u32", "u64", "f32", "f64", "i32", "i64"])
@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("n", [1, 33, 6144 * 5 + 77, 1 << 20])
def test_descending_matches_oracle(kt, pairs, n):
    _dev()
    keys = _keys(kt, "and2" if n > 1000 else "uniform", n, seed=n + KB[kt])
    vals = workload.iota_u32(n) if pairs else None
    k = _to_dev(keys)
    if pairs:
        ko, vo = osw.sort_pairs(k, _to_dev(vals), key_type=kt, descending=True)
        torch.cuda.synchronize()
        ek, ev = oracle.sort(kt, keys, vals, descending=True)
        assert np.array_equal(ko.cpu().numpy().view(_kd(kt)), ek)
        assert np.array_equal(vo.cpu().numpy().view(np.uint32), ev)
    else:
        ko = osw.sort_keys(k, key_type=kt, descending=True)
        torch.cuda.synchronize()
        assert np.array_equal(ko.cpu().numpy().view(_kd(kt)), oracle.sort(kt, keys, descending=True))


@pytest.mark.parametrize("kt,begin,end", [("u32", 3, 29), ("u32", 0, 8), ("u64", 5, 50), ("i32", 0, 32),
                                          ("i64", 7, 64), ("f32", 0, 32)])
@pytest.mark.parametrize("dist", ["and3", "const", "and16"])
def test_descending_bit_ranges_and_distributions(kt, begin, end, dist):
    _dev()
    n = 300_007
    keys = _keys(kt, dist, n, seed=begin * 97 + end)
    vals = workload.iota_u32(n)
    ko, vo = osw.sort_pairs(_to_dev(keys), _to_dev(vals), begin, end, key_type=kt, descending=True)
    torch.cuda.synchronize()
    ek, ev = oracle.sort(kt, keys, vals, begin, end, descending=True)
    assert np.array_equal(ko.cpu().numpy().view(_kd(kt)), ek)
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), ev)


@pytest.mark.parametrize("cfg", list(range(12)))
def test_descending_every_tile_config(cfg):
    _dev()
    prev = osw.os_get_tile_config(32, 4)
    try:
        assert osw.os_set_tile_config(32, 4, cfg) == osw.OS_OK
        t = osw.os_tile_config_keys(32, 4, cfg)
        n = 3 * t + 5
        keys = _keys("u32", "and2", n, seed=cfg)
        vals = workload.iota_u32(n)
        ko, vo = osw.sort_pairs(_to_dev(keys), _to_dev(vals), key_type="u32", descending=True)
        torch.cuda.synchronize()
        ek, ev = oracle.sort("u32", keys, vals, descending=True)
        assert np.array_equal(ko.cpu().numpy().view(np.uint32), ek)
        assert np.array_equal(vo.cpu().numpy().view(np.uint32), ev)
    finally:
        osw.os_set_tile_config(32, 4, prev)


@pytest.mark.parametrize("kt", ["u32", "i64", "f32"])
def test_descending_histograms_and_offsets(kt):
    _dev()
    n = 100_003
    keys = _keys(kt, "uniform", n, seed=5)
    h, o = osw.digit_histograms(_to_dev(keys), 0, KB[kt] - 3, key_type=kt, descending=True)
    torch.cuda.synchronize()
    assert np.array_equal(h.cpu().numpy().astype(np.uint64), oracle.histograms(kt, keys, 0, KB[kt] - 3,
                                                                              descending=True))
    assert np.array_equal(o.cpu().numpy().astype(np.uint64), oracle.bin_offsets(kt, keys, 0, KB[kt] - 3,
                                                                               descending=True))


@pytest.mark.parametrize("kt", ["u32", "u64", "f32"])
def test_descending_batch(kt):
    _dev()
    rng = np.random.default_rng(3)
    # empty, one-key, small (one-block path) and multi-tile segments
    sizes = [0, 1, 5, 1000, 4096, 4097, 20_000, 70_001] + list(rng.integers(0, 3000, 40))
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offs[-1])
    keys = _keys(kt, "and2", n, seed=11)
    vals = workload.iota_u32(n)
    ko, vo = osw.sort_batch(_to_dev(keys), torch.from_numpy(offs).to(_dev()), _to_dev(vals), key_type=kt,
                            descending=True)
    torch.cuda.synchronize()
    ek, ev = oracle.sort_segments(kt, keys, offs.astype(np.uint64), vals, descending=True)
    assert np.array_equal(ko.cpu().numpy().view(_kd(kt)), ek)
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), ev)


def test_descending_host_buffers_and_unknown_flags():
    _dev()
    n = 50_001
    keys = _keys("u64", "uniform", n, seed=8)
    vals = workload.iota_u32(n)
    ko, vo = osw.sort_host(keys, vals, key_type="u64", descending=True)
    ek, ev = oracle.sort("u64", keys, vals, descending=True)
    assert np.array_equal(np.asarray(ko).view(np.uint64), ek) and np.array_equal(np.asarray(vo).view(np.uint32), ev)
    # a key type with an unknown flag bit is refused
    assert osw.os_sort_workspace_bytes(osw.OS_KEY_U32 | 0x200, 100, 0, 0, 32) == 0
    assert osw.os_sort_workspace_bytes(osw.OS_KEY_U32 | osw.OS_SORT_DESCENDING, 100, 0, 0, 32) > 0
