"""GPU parity: the CUDA path through the C ABI against the CPU oracle, bit-exact.

Every input is seeded and synthetic (``paper_2206_01784_gb300.workload``); the
oracle sees the same bits. Sizes span several tiles with ragged tails, plus
the edge cases: empty, single key, one short tile, exact multiples of the
tile, unaligned pointers, narrow and odd bit ranges, all-equal keys.
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


def to_dev(a: np.ndarray, offset: int = 0):
    """numpy uint32/uint64 -> CUDA tensor of the same bits (optionally at an
    element offset inside a larger buffer, to get an unaligned pointer)."""
    view = a.view(np.int64 if a.dtype.itemsize == 8 else np.int32)
    if offset == 0:
        return torch.from_numpy(view.copy()).to(_dev())
    buf = torch.empty(a.size + offset, dtype=torch.int64 if a.dtype.itemsize == 8 else torch.int32, device=_dev())
    buf[offset:] = torch.from_numpy(view.copy()).to(_dev())
    return buf[offset:]


def to_host(t, dtype):
    return t.cpu().numpy().view(dtype)


def kdtype(kt):
    return np.uint64 if KB[kt] == 64 else np.uint32


def tile_keys(kt, pairs):
    return osw.os_sort_workspace_layout(osw.KEY_TYPES[kt], 1, 4 if pairs else 0, 0, KB[kt]).tile_keys


def gpu_sort(kt, keys_np, vals_np=None, begin=0, end=None, offset=0):
    end = KB[kt] if end is None else end
    k = to_dev(keys_np, offset)
    if vals_np is None:
        out = osw.sort_keys(k, begin, end, key_type=kt)
        torch.cuda.synchronize()
        return to_host(out, kdtype(kt))
    v = to_dev(vals_np, offset)
    ko, vo = osw.sort_pairs(k, v, begin, end, key_type=kt)
    torch.cuda.synchronize()
    return to_host(ko, kdtype(kt)), to_host(vo, np.uint32)


def make_keys(kt, dist, n, seed):
    if kt in ("f32", "f64") and dist == "uniform":
        dist = "normal"
    return workload.keys(kt, dist, n, seed)


def test_loaded_device_code_is_sm103():
    _dev()
    assert osw.os_binary_version() == 103


# ---------------------------------------------------------------- phase 1 + 2

@pytest.mark.parametrize("kt,begin,end", [("u32", 0, 32), ("u32", 3, 29), ("u64", 0, 64), ("u64", 5, 50),
                                          ("f32", 0, 32), ("f64", 0, 64), ("u32", 0, 8), ("i32", 0, 32),
                                          ("i64", 3, 64)])
@pytest.mark.parametrize("n", [1, 3, 31, 33, 4097, 100_003, 1 << 20])
def test_histograms_and_offsets(kt, begin, end, n):
    keys = make_keys(kt, "uniform", n, seed=n)
    h, o = osw.digit_histograms(to_dev(keys), begin, end, key_type=kt)
    torch.cuda.synchronize()
    assert np.array_equal(h.cpu().numpy().astype(np.uint64), oracle.histograms(kt, keys, begin, end))
    assert np.array_equal(o.cpu().numpy().astype(np.uint64), oracle.bin_offsets(kt, keys, begin, end))


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_histograms_unaligned(offset):
    keys = make_keys("u32", "and2", 70_001, seed=3)
    h, o = osw.digit_histograms(to_dev(keys, offset), 0, 32, key_type="u32")
    torch.cuda.synchronize()
    assert np.array_equal(h.cpu().numpy().astype(np.uint64), oracle.histograms("u32", keys))


# ---------------------------------------------------------------- one binning pass

@pytest.mark.parametrize("kt", ["u32", "u64", "f32"])
@pytest.mark.parametrize("pairs", [False, True])
def test_single_pass(kt, pairs):
    t = tile_keys(kt, pairs)
    n = 5 * t + 77
    keys = make_keys(kt, "uniform", n, seed=17)
    vals = workload.iota_u32(n) if pairs else None
    for begin in (0, 8, KB[kt] - 8):
        got = gpu_sort(kt, keys, vals, begin, begin + 8)
        exp = oracle.sort(kt, keys, vals, begin, begin + 8)
        if pairs:
            assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])
        else:
            assert np.array_equal(got, exp)


def test_lookback_final_status_counters():
    # After a one-pass sort every status counter holds (G, inclusive prefix of
    # its digit's per-tile counts) - the final state of Figure 7 (f).
    kt, n = "u32", None
    lay0 = osw.os_sort_workspace_layout(osw.OS_KEY_U32, 1, 0, 0, 8)
    t = lay0.tile_keys
    n = 9 * t + 1234
    keys = make_keys(kt, "and2", n, seed=23)
    lay = osw.os_sort_workspace_layout(osw.OS_KEY_U32, n, 0, 0, 8)
    ws = torch.empty(lay.total_bytes, dtype=torch.uint8, device=_dev())
    k = to_dev(keys)
    out = torch.empty_like(k)
    s = torch.cuda.current_stream().cuda_stream
    rc = osw.os_sort_keys(osw.OS_KEY_U32, k.data_ptr(), out.data_ptr(), n, 0, 8, ws.data_ptr(), ws.numel(), s)
    assert rc == osw.OS_OK
    assert osw.os_workspace_status(ws.data_ptr(), s) == osw.OS_OK
    slab = ws[lay.status_offset[0]: lay.status_offset[0] + lay.num_tiles * 256 * 4].cpu().numpy().view(np.uint32)
    slab = slab.reshape(lay.num_tiles, 256)
    counts = oracle.tile_digit_counts(kt, keys, 0, 8, t)
    inclusive = np.cumsum(counts, axis=0)
    assert np.all(slab >> 30 == 2)
    assert np.array_equal((slab & ((1 << 30) - 1)).astype(np.uint64), inclusive)


# ---------------------------------------------------------------- full sorts

SIZES = [1, 2, 31, 32, 33, 1000]


@pytest.mark.parametrize("kt", ["u32", "u64", "f32", "f64", "i32", "i64"])
@pytest.mark.parametrize("pairs", [False, True])
def test_sort_edge_sizes(kt, pairs):
    t = tile_keys(kt, pairs)
    for n in SIZES + [t - 1, t, t + 1, 3 * t, 3 * t + 5]:
        keys = make_keys(kt, "uniform", n, seed=n + 1)
        vals = workload.iota_u32(n) if pairs else None
        got = gpu_sort(kt, keys, vals)
        exp = oracle.sort(kt, keys, vals)
        if pairs:
            assert np.array_equal(got[0], exp[0]), n
            assert np.array_equal(got[1], exp[1]), n
        else:
            assert np.array_equal(got, exp), n


def test_sort_empty():
    k = torch.empty(0, dtype=torch.int32, device=_dev())
    out = osw.sort_keys(k, key_type="u32")
    assert out.numel() == 0


@pytest.mark.parametrize("dist", ["uniform", "and2", "and3", "and4", "and5", "and8", "and16", "const"])
@pytest.mark.parametrize("kt", ["u32", "u64"])
def test_sort_distributions(dist, kt):
    n = (1 << 20) + 12345
    keys = make_keys(kt, dist, n, seed=5)
    vals = workload.iota_u32(n)
    got = gpu_sort(kt, keys, vals)
    exp = oracle.sort(kt, keys, vals)
    assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])


@pytest.mark.parametrize("kt", ["f32", "f64"])
def test_sort_float_normal(kt):
    n = (1 << 20) + 3
    keys = make_keys(kt, "normal", n, seed=9)
    vals = workload.iota_u32(n)
    got = gpu_sort(kt, keys, vals)
    exp = oracle.sort(kt, keys, vals)
    assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])


def test_sort_float_specials():
    sp = np.array([0x7F800000, 0xFF800000, 0x7FC00000, 0xFFC00000, 0x80000000, 0x00000000, 0x00000001,
                   0x80000001, 0x7F7FFFFF, 0xFF7FFFFF], np.uint32)
    keys = np.tile(sp, 5000)
    vals = workload.iota_u32(keys.size)
    got = gpu_sort("f32", keys, vals)
    exp = oracle.sort("f32", keys, vals)
    assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])


@pytest.mark.parametrize("kt,begin,end", [("u32", 0, 0), ("u32", 4, 20), ("u32", 13, 31), ("u32", 7, 8),
                                          ("u64", 5, 50), ("u64", 0, 33), ("f32", 16, 32), ("u64", 60, 64),
                                          ("i32", 0, 32), ("i32", 5, 32), ("i32", 3, 31), ("i64", 0, 64),
                                          ("i64", 7, 64), ("i64", 0, 40)])
def test_sort_bit_ranges(kt, begin, end):
    n = 3 * tile_keys(kt, True) + 99
    keys = make_keys(kt, "uniform", n, seed=begin * 100 + end)
    vals = workload.iota_u32(n)
    got = gpu_sort(kt, keys, vals, begin, end)
    exp = oracle.sort(kt, keys, vals, begin, end)
    assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])


@pytest.mark.parametrize("offset", [1, 3])
@pytest.mark.parametrize("kt", ["u32", "u64"])
def test_sort_unaligned_pointers(offset, kt):
    n = 4 * tile_keys(kt, True) + 17
    keys = make_keys(kt, "and2", n, seed=31)
    vals = workload.iota_u32(n)
    got = gpu_sort(kt, keys, vals, offset=offset)
    exp = oracle.sort(kt, keys, vals)
    assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])


def test_inputs_preserved_and_repeatable():
    n = 300_001
    keys = make_keys("u32", "uniform", n, seed=41)
    vals = workload.iota_u32(n)
    k, v = to_dev(keys), to_dev(vals)
    ws = osw.workspace(osw.OS_KEY_U32, n, 4, 0, 32, k.device)
    a = osw.sort_pairs(k, v, ws=ws, key_type="u32")
    b = osw.sort_pairs(k, v, ws=ws, key_type="u32")
    torch.cuda.synchronize()
    assert np.array_equal(to_host(k, np.uint32), keys) and np.array_equal(to_host(v, np.uint32), vals)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_stream_argument():
    _dev()
    n = 200_000
    keys = make_keys("u32", "uniform", n, seed=43)
    s = torch.cuda.Stream()
    k = to_dev(keys)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        out = osw.sort_keys(k, key_type="u32", stream=s)
    s.synchronize()
    assert np.array_equal(to_host(out, np.uint32), oracle.sort("u32", keys))


# ---------------------------------------------------------------- failure detection

def test_lookback_wait_limit_reports_timeout():
    # A tile that never publishes makes its successors' waits run out; the
    # device records it and os_workspace_status returns OS_ERR_TIMEOUT. The
    # context stays usable and the next sort is correct.
    n = 6 * tile_keys("u32", False) + 5
    keys = make_keys("u32", "uniform", n, seed=47)
    k = to_dev(keys)
    ws = osw.workspace(osw.OS_KEY_U32, n, 0, 0, 32, k.device)
    s = torch.cuda.current_stream().cuda_stream
    out = torch.empty_like(k)
    try:
        osw.os_debug_set_lookback_fault(2, 1 << 14)
        rc = osw.os_sort_keys(osw.OS_KEY_U32, k.data_ptr(), out.data_ptr(), n, 0, 32, ws.data_ptr(), ws.numel(), s)
        assert rc == osw.OS_OK
        assert osw.os_workspace_status(ws.data_ptr(), s) == osw.OS_ERR_TIMEOUT
    finally:
        osw.os_debug_set_lookback_fault(-1, 0)
    rc = osw.os_sort_keys(osw.OS_KEY_U32, k.data_ptr(), out.data_ptr(), n, 0, 32, ws.data_ptr(), ws.numel(), s)
    assert rc == osw.OS_OK
    assert osw.os_workspace_status(ws.data_ptr(), s) == osw.OS_OK
    assert np.array_equal(to_host(out, np.uint32), oracle.sort("u32", keys))


@pytest.mark.parametrize("cfg", list(range(12)))
@pytest.mark.parametrize("kt", ["u32", "u64", "f32"])
def test_every_tile_config(cfg, kt):
    # every binning variant (three one-block-per-tile geometries and the
    # persistent kernel, each with three ranking methods) gives the oracle's
    # result (workspaces are sized for the smallest tile, so the same sizing
    # serves all of them)
    assert osw.os_num_tile_configs() == 12
    kb = KB[kt]
    prev = {vb: osw.os_get_tile_config(kb, vb) for vb in (0, 4)}
    try:
        for pairs in (False, True):
            assert osw.os_set_tile_config(kb, 4 if pairs else 0, cfg) == osw.OS_OK
            t = osw.os_tile_config_keys(kb, 4 if pairs else 0, cfg)
            for n in (t - 1, 2 * t, 5 * t + 3):
                keys = make_keys(kt, "and2" if kt != "f32" else "normal", n, seed=cfg * 7 + n)
                vals = workload.iota_u32(n) if pairs else None
                got = gpu_sort(kt, keys, vals)
                exp = oracle.sort(kt, keys, vals)
                if pairs:
                    assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1]), (cfg, n)
                else:
                    assert np.array_equal(got, exp), (cfg, n)
    finally:
        for vb in (0, 4):
            osw.os_set_tile_config(kb, vb, prev[vb])


def test_autotune_small_buckets_keeps_results():
    from paper_2206_01784_gb300 import autotune

    _dev()
    saved = autotune.current()
    try:
        table = autotune.tune(key_bits=(32,), value_bytes=(4,), buckets=(0, 1), steps=2, warmup=1)
        for b in (0, 1):
            rec = table[(32, 4, b)]
            # every variant with 8-bit digits, variant 4 with 5-, 6- and 7-bit digits
            assert len(rec["ms"]) == osw.os_num_tile_configs() + 3 and all(t > 0 for t in rec["ms"].values())
            assert osw.os_get_tile_config_bucket(32, 4, b) == rec["cfg"]
            assert osw.os_get_radix_bits_bucket(32, 4, b) == rec["radix_bits"]
        n = 300_007
        keys = make_keys("u32", "and2", n, seed=99)
        vals = workload.iota_u32(n)
        got = gpu_sort("u32", keys, vals)
        exp = oracle.sort("u32", keys, vals)
        assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])
    finally:
        autotune.apply(saved)
