"""Strips (Section 3, "Handling very large problems"): passes over 2^30 keys
or more run as one chained scan per strip (strips of equal length, each below
2^30 keys), each strip's bins starting where the previous strip's ended.

The multi-strip path is exercised here on small inputs with the shortest
strip limit the library allows (2^16 keys), bit-exact against the oracle; the
slow cases run 2^28 + 12345 uint32 pairs in 2^26-key strips against the
oracle, and 2^30 + 12345 uint32 pairs (two strips at the default limit) by
the properties that pin the stable sort.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2206_01784_gb300 import onesweep as osw  # noqa: E402
from paper_2206_01784_gb300 import workload  # noqa: E402

pytestmark = pytest.mark.gpu

KB = {"u32": 32, "u64": 64, "f32": 32, "f64": 64, "i32": 32, "i64": 64}
SHORT = 1 << 16


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _to_dev(a):
    return torch.from_numpy(a.view(np.int64 if a.dtype.itemsize == 8 else np.int32).copy()).to(_dev())


def _host(t, dt):
    return t.cpu().numpy().view(dt)


@pytest.fixture
def short_strips():
    _dev()
    assert osw.os_debug_set_strip_keys(SHORT) == SHORT
    try:
        yield SHORT
    finally:
        osw.os_debug_set_strip_keys(0)


def _strip_len(kt, pairs, n_hint=4 * SHORT):
    # the strip limit in whole tiles of a sort of about n_hint keys (the
    # geometry depends on size); the library then balances the strips
    tile = osw.os_sort_workspace_layout(osw.KEY_TYPES[kt], n_hint, 4 if pairs else 0, 0, KB[kt]).tile_keys
    return SHORT // tile * tile


def _keys(kt, dist, n, seed):
    if kt in ("f32", "f64") and dist == "uniform":
        dist = "normal"
    return workload.keys(kt, dist, n, seed)


def _sort(kt, keys, vals, begin, end):
    dt = np.uint64 if KB[kt] == 64 else np.uint32
    if vals is None:
        out = osw.sort_keys(_to_dev(keys), begin, end, key_type=kt)
        torch.cuda.synchronize()
        return _host(out, dt)
    ko, vo = osw.sort_pairs(_to_dev(keys), _to_dev(vals), begin, end, key_type=kt)
    torch.cuda.synchronize()
    return _host(ko, dt), _host(vo, np.uint32)


def _check(got, exp, pairs):
    if pairs:
        assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])
    else:
        assert np.array_equal(got, exp)


@pytest.mark.parametrize("kt,pairs", [("u32", True), ("u32", False), ("u64", True), ("u64", False),
                                      ("f32", True), ("f64", False), ("i32", True), ("i64", True)])
@pytest.mark.parametrize("dist", ["uniform", "and4", "const"])
def test_short_strips_exact(short_strips, kt, pairs, dist):
    strip = _strip_len(kt, pairs)
    n = 4 * strip + 777  # five strips, the last one ragged
    keys = _keys(kt, dist, n, seed=101)
    vals = workload.iota_u32(n) if pairs else None
    _check(_sort(kt, keys, vals, 0, KB[kt]), oracle.sort(kt, keys, vals, 0, KB[kt]), pairs)


@pytest.mark.parametrize("kt,begin,end", [("u32", 3, 29), ("u64", 5, 50), ("i64", 7, 64), ("u32", 0, 8)])
def test_short_strips_bit_ranges(short_strips, kt, begin, end):
    strip = _strip_len(kt, True)
    n = 3 * strip + 4099
    keys = _keys(kt, "uniform", n, seed=103)
    vals = workload.iota_u32(n)
    _check(_sort(kt, keys, vals, begin, end), oracle.sort(kt, keys, vals, begin, end), True)


def test_short_strips_boundaries(short_strips):
    # exactly the strip limit, one key past it (two half strips), an exact
    # multiple of it, one key short of two
    strip = _strip_len("u32", True)
    for n in (strip, strip + 1, 3 * strip, 2 * strip - 1):
        keys = _keys("u32", "and2", n, seed=n)
        vals = workload.iota_u32(n)
        _check(_sort("u32", keys, vals, 0, 32), oracle.sort("u32", keys, vals, 0, 32), True)


def test_short_strips_every_tile_config(short_strips):
    prev = osw.os_get_tile_config(32, 4)
    try:
        for cfg in range(osw.os_num_tile_configs()):
            assert osw.os_set_tile_config(32, 4, cfg) == osw.OS_OK
            strip = _strip_len("u32", True)
            n = 2 * strip + 5003
            keys = _keys("u32", "uniform", n, seed=200 + cfg)
            vals = workload.iota_u32(n)
            _check(_sort("u32", keys, vals, 0, 32), oracle.sort("u32", keys, vals, 0, 32), True)
    finally:
        osw.os_set_tile_config(32, 4, prev)


def test_workspace_sized_once_fits_short_strips():
    # a workspace sized under the default strip length serves a sort with
    # short strips (more tile counters) without growing
    dev = _dev()
    n = 7 * SHORT + 3
    bytes_default = osw.os_sort_workspace_bytes(osw.OS_KEY_U32, n, 4, 0, 32)
    osw.os_debug_set_strip_keys(SHORT)
    try:
        assert osw.os_sort_workspace_bytes(osw.OS_KEY_U32, n, 4, 0, 32) == bytes_default
        keys = _keys("u32", "uniform", n, seed=5)
        vals = workload.iota_u32(n)
        k, v = _to_dev(keys), _to_dev(vals)
        ko, vo = torch.empty_like(k), torch.empty_like(v)
        ws = torch.empty(bytes_default, dtype=torch.uint8, device=dev)
        s = torch.cuda.current_stream().cuda_stream
        rc = osw.os_sort_pairs(osw.OS_KEY_U32, k.data_ptr(), ko.data_ptr(), v.data_ptr(), vo.data_ptr(), n, 0, 32,
                               ws.data_ptr(), ws.numel(), s)
        assert rc == osw.OS_OK and osw.os_workspace_status(ws.data_ptr(), s) == osw.OS_OK
        exp = oracle.sort("u32", keys, vals, 0, 32)
        assert np.array_equal(_host(ko, np.uint32), exp[0]) and np.array_equal(_host(vo, np.uint32), exp[1])
    finally:
        osw.os_debug_set_strip_keys(0)


@pytest.mark.slow
def test_large_strips_exact():
    _dev()
    n = (1 << 28) + 12345  # five strips of 2^26 keys or less
    keys = workload.keys("u32", "uniform", n, 11)
    vals = workload.iota_u32(n)
    osw.os_debug_set_strip_keys(1 << 26)
    try:
        got = _sort("u32", keys, vals, 0, 32)
    finally:
        osw.os_debug_set_strip_keys(0)
    exp = oracle.sort("u32", keys, vals, 0, 32)
    assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])


@pytest.mark.slow
def test_beyond_2_30_keys_by_properties():
    # n past the 30-bit count limit of one chained scan: two strips per pass.
    # Properties that hold exactly for the stable sort, checked on the host.
    _dev()
    n = (1 << 30) + 12345
    keys = workload.keys("u32", "and2", n, 12)
    ko, vo = _sort("u32", keys, workload.iota_u32(n), 0, 32)
    assert np.all(ko[1:] >= ko[:-1]), "not sorted"
    seen = np.zeros(n, dtype=bool)
    seen[vo] = True
    assert seen.all(), "values are not a permutation"
    del seen
    assert np.array_equal(keys[vo], ko), "keys do not follow their values"
    eq = ko[1:] == ko[:-1]
    assert np.all(vo[1:][eq] > vo[:-1][eq]), "not stable"
