"""Digit widths other than 8 bits (os_sort_options.radix_bits = 5..7), against the oracle.

Section 4's Table 2 measures the same sort with d = 5..9 bits per digit place.
The sorted output does not depend on d; the passes do, so besides whole
sorts the tests pin one pass of d-bit digits against the oracle's first pass
with the same digit width.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2206_01784_gb300 import onesweep as osw, workload

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
_INT = {"u32": np.int32, "i32": np.int32, "f32": np.int32, "u64": np.int64, "i64": np.int64, "f64": np.int64}


def _dev(a, kt):
    return torch.from_numpy(a.view(_INT[kt]).copy()).to(DEV)


def _vals(n):
    return torch.from_numpy(workload.iota_u32(n).view(np.int32).copy()).to(DEV)


@pytest.mark.parametrize("d", [5, 6, 7, 8])
@pytest.mark.parametrize("kt,dist,n,pairs", [
    ("u32", "uniform", (1 << 20) + 77, True),
    ("u32", "uniform", 1000003, False),
    ("u32", "and3", 300001, True),
    ("u32", "const", 100000, True),
    ("u64", "uniform", 250001, True),
    ("f32", "normal", 400003, True),
    ("i64", "uniform", 70001, False),
    ("i32", "uniform", 6143, True),
])
def test_sort_with_digit_width(d, kt, dist, n, pairs):
    keys = workload.keys(kt, dist, n, seed=n % 101 + d)
    k = _dev(keys, kt)
    if pairs:
        vals = workload.iota_u32(n)
        ko, vo = osw.sort_pairs(k, _vals(n), key_type=kt, radix_bits=d)
        ek, ev = oracle.sort(kt, keys, vals)
        assert np.array_equal(vo.cpu().numpy().view(np.uint32), ev)
    else:
        ko = osw.sort_keys(k, key_type=kt, radix_bits=d)
        ek = oracle.sort(kt, keys)
    assert np.array_equal(ko.cpu().numpy().view(ek.dtype), ek)


@pytest.mark.parametrize("d", [5, 6, 7])
@pytest.mark.parametrize("begin,end,desc", [(3, 29, False), (0, 32, True), (7, 8, False), (0, 17, True)])
def test_bit_ranges_and_order(d, begin, end, desc):
    n = 200003
    for kt in ("u32", "i32"):
        keys = workload.keys(kt, "uniform", n, seed=begin * 7 + end + d)
        vals = workload.iota_u32(n)
        ko, vo = osw.sort_pairs(_dev(keys, kt), _vals(n), begin_bit=begin, end_bit=end, key_type=kt,
                                descending=desc, radix_bits=d)
        ek, ev = oracle.sort(kt, keys, vals, begin_bit=begin, end_bit=end, descending=desc)
        assert np.array_equal(ko.cpu().numpy().view(ek.dtype), ek)
        assert np.array_equal(vo.cpu().numpy().view(np.uint32), ev)


@pytest.mark.parametrize("d", [5, 6, 7, 8])
def test_one_pass_matches_oracle_pass(d):
    # a sort over bits [0, d) with d-bit digits is exactly one binning pass
    n = (1 << 19) + 5
    keys = workload.keys("u32", "uniform", n, seed=40 + d)
    vals = workload.iota_u32(n)
    ko, vo = osw.sort_pairs(_dev(keys, "u32"), _vals(n), begin_bit=0, end_bit=d, key_type="u32", radix_bits=d)
    ek, ev = oracle.sort("u32", keys, vals, radix_bits=d, passes=1)
    assert np.array_equal(ko.cpu().numpy().view(np.uint32), ek)
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), ev)


def test_thirteen_places_fit_the_workspace():
    # 64-bit keys in 5-bit digits: 13 passes, on a workspace sized without d
    n = 123457
    keys = workload.keys("u64", "and2", n, seed=3)
    vals = workload.iota_u32(n)
    ws = osw.workspace(osw.KEY_TYPES["u64"], n, 4, 0, 64, DEV)
    ko, vo = osw.sort_pairs(_dev(keys, "u64"), _vals(n), key_type="u64", ws=ws, radix_bits=5)
    ek, ev = oracle.sort("u64", keys, vals)
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), ek)
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), ev)


def test_invalid_digit_widths_rejected():
    n = 4096
    k = torch.zeros(n, dtype=torch.int32, device=DEV)
    out = torch.empty_like(k)
    ws = osw.workspace(osw.KEY_TYPES["u32"], n, 0, 0, 32, DEV)
    s = torch.cuda.current_stream().cuda_stream
    call = lambda **kw: osw.os_sort_keys_ex(osw.KEY_TYPES["u32"], k.data_ptr(), out.data_ptr(), n, 0, 32,  # noqa
                                            ws.data_ptr(), ws.numel(), s, **kw)
    for bad in (1, 4, 9, 16):
        assert call(radix_bits=bad) == osw.OS_ERR_INVALID_ARG
    assert call(radix_bits=6, tile_config=0) == osw.OS_ERR_INVALID_ARG   # narrow digits run variant 4
    assert call(radix_bits=6, tile_config=4) == osw.OS_OK
    assert call(radix_bits=6) == osw.OS_OK
    assert call(radix_bits=0) == osw.OS_OK
    torch.cuda.synchronize()
    # batches bin 8-bit digits only
    offs = torch.tensor([0, n], dtype=torch.int64, device=DEV)
    bws = osw.batch_workspace(osw.KEY_TYPES["u32"], n, 1, 0, 0, 32, DEV)
    rc = osw.os_sort_batch_ex(osw.KEY_TYPES["u32"], k.data_ptr(), out.data_ptr(), None, None, offs.data_ptr(), 1, n,
                              0, 32, bws.data_ptr(), bws.numel(), s, radix_bits=6)
    assert rc == osw.OS_ERR_INVALID_ARG


def test_process_wide_width_used_when_options_leave_it_open():
    n = 300001
    kb, vb = 32, 4
    bucket = osw.os_size_bucket(n)
    saved = osw.os_get_radix_bits_bucket(kb, vb, bucket)
    keys = workload.keys("u32", "uniform", n, seed=77)
    vals = workload.iota_u32(n)
    try:
        assert osw.os_set_radix_bits_bucket(kb, vb, bucket, 6) == osw.OS_OK
        torch.cuda.synchronize()
        osw.os_profile_start(64)
        ko, vo = osw.sort_pairs(_dev(keys, "u32"), _vals(n), key_type="u32")
        torch.cuda.synchronize()
        _, _, recs = osw.os_profile_stop(64)
        # 32 bits in 6-bit digits: 6 binning passes after the one histogram launch
        assert sum(1 for k, _, _ in recs if k == 1) == 6
        assert sum(1 for k, _, _ in recs if k == 0) == 1
        ek, ev = oracle.sort("u32", keys, vals)
        assert np.array_equal(ko.cpu().numpy().view(np.uint32), ek)
        assert np.array_equal(vo.cpu().numpy().view(np.uint32), ev)
        # a call that names another tile variant keeps 8-bit digits
        osw.os_profile_start(64)
        k, v = _dev(keys, "u32"), _vals(n)
        out, vout = torch.empty_like(k), torch.empty_like(v)
        ws = osw.workspace(osw.KEY_TYPES["u32"], n, 4, 0, 32, DEV)
        assert osw.os_sort_pairs_ex(osw.KEY_TYPES["u32"], k.data_ptr(), out.data_ptr(), v.data_ptr(), vout.data_ptr(),
                                    n, 0, 32, ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream,
                                    tile_config=0) == osw.OS_OK
        torch.cuda.synchronize()
        _, _, recs = osw.os_profile_stop(64)
        assert sum(1 for k_, _, _ in recs if k_ == 1) == 4
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ek)
        assert np.array_equal(vout.cpu().numpy().view(np.uint32), ev)
    finally:
        osw.os_set_radix_bits_bucket(kb, vb, bucket, saved)
