"""os_sort_noalloc: the sort for callers that cannot allocate device memory.

Such callers (code whose device memory belongs to another allocator, or that
must not trigger the implicit device synchronization of cudaMalloc/cudaFree)
hand over only their inputs and outputs; the scratch comes from a fixed
16 MiB array of static device memory in the library. These tests call the
entry point through the C ABI twice in a row on different inputs (the second
call finds the first one's leftovers in the shared scratch) and require the
output of each call to equal, bit for bit, both the regular entry point's
(os_sort_pairs / os_sort_keys, which take a caller-allocated workspace) and
the CPU oracle's. They also check that a sort too large for the fixed
scratch is refused, and that argument errors are named first.

This file is collected last so that, if it fails, a run stopping at the first
failure has already run every other test. It passes alone in a fresh process
and after the rest of the suite.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2206_01784_gb300 import onesweep as osw  # noqa: E402
from paper_2206_01784_gb300 import workload  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _to_dev(a):
    return torch.from_numpy(a.view(np.int64 if a.dtype.itemsize == 8 else np.int32).copy()).to(_dev())


def _regular(kt, k, v, n, begin, end, s):
    """The existing entry point with a caller-allocated workspace."""
    ws = osw.workspace(kt, n, 4 if v is not None else 0, begin, end, k.device)
    ko = torch.empty_like(k)
    if v is None:
        rc = osw.os_sort_keys(kt, k.data_ptr(), ko.data_ptr(), n, begin, end, ws.data_ptr(), ws.numel(), s)
        vo = None
    else:
        vo = torch.empty_like(v)
        rc = osw.os_sort_pairs(kt, k.data_ptr(), ko.data_ptr(), v.data_ptr(), vo.data_ptr(), n, begin, end,
                               ws.data_ptr(), ws.numel(), s)
    assert rc == osw.OS_OK
    assert osw.os_workspace_status(ws.data_ptr(), s) == osw.OS_OK
    return ko, vo


def _noalloc(kt, k, v, n, begin, end, s):
    ko = torch.empty_like(k)
    vo = torch.empty_like(v) if v is not None else None
    rc, scratch = osw.os_sort_noalloc(kt, k.data_ptr(), ko.data_ptr(), None if v is None else v.data_ptr(),
                                      None if v is None else vo.data_ptr(), n, begin, end, s)
    assert rc == osw.OS_OK, osw.os_status_string(rc)
    assert scratch
    assert osw.os_workspace_status(scratch, s) == osw.OS_OK
    return ko, vo


CASES = [
    ("u32", True, 1 << 20, 0, 32),       # the largest size that always fits
    ("u32", False, 300_001, 0, 32),
    ("f32", True, 123_457, 0, 32),
    ("u64", True, (1 << 20) - 3, 0, 64),
    ("u32", True, 77_777, 3, 29),
    ("u32", True, 1, 0, 32),
]


@pytest.mark.parametrize("kt,pairs,n,begin,end", CASES)
def test_noalloc_matches_regular_entry_point_twice(kt, pairs, n, begin, end):
    _dev()
    key_type = osw.KEY_TYPES[kt]
    s = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((101, 202)):  # two calls in a row share the static scratch
        dist = "normal" if kt == "f32" else ("and2" if call else "uniform")
        keys = workload.keys(kt, dist, n, seed + n)
        k = _to_dev(keys)
        v = _to_dev(workload.iota_u32(n)) if pairs else None
        rk, rv = _regular(key_type, k, v, n, begin, end, s)
        nk, nv = _noalloc(key_type, k, v, n, begin, end, s)
        torch.cuda.synchronize()
        assert torch.equal(nk, rk), (kt, n, call)
        if pairs:
            assert torch.equal(nv, rv), (kt, n, call)
        # and element by element against the CPU oracle
        kd = np.uint64 if keys.dtype.itemsize == 8 else np.uint32
        got_k = nk.cpu().numpy().view(kd)
        if pairs:
            ek, ev = oracle.sort(kt, keys, workload.iota_u32(n), begin, end)
            assert np.array_equal(got_k, ek), (kt, n, call)
            assert np.array_equal(nv.cpu().numpy().view(np.uint32), ev), (kt, n, call)
        else:
            assert np.array_equal(got_k, oracle.sort(kt, keys, None, begin, end)), (kt, n, call)


def test_noalloc_rejects_sorts_beyond_its_scratch():
    _dev()
    n = 1 << 23  # its workspace is far above 16 MiB
    k = torch.empty(n, dtype=torch.int32, device=_dev())
    v = torch.empty_like(k)
    ko, vo = torch.empty_like(k), torch.empty_like(v)
    s = torch.cuda.current_stream().cuda_stream
    rc, _ = osw.os_sort_noalloc(osw.OS_KEY_U32, k.data_ptr(), ko.data_ptr(), v.data_ptr(), vo.data_ptr(), n, 0, 32, s)
    assert rc == osw.OS_ERR_SCRATCH_LIMIT
    assert "16 MiB" in osw.os_status_string(rc)
    # argument errors are still named as by the regular entry point, before
    # the scratch limit: a bad bit range, one value pointer without the other
    rc, _ = osw.os_sort_noalloc(osw.OS_KEY_U32, k.data_ptr(), ko.data_ptr(), None, None, 1000, 0, 33, s)
    assert rc == osw.OS_ERR_INVALID_ARG
    rc, _ = osw.os_sort_noalloc(osw.OS_KEY_U32, k.data_ptr(), ko.data_ptr(), v.data_ptr(), None, n, 0, 32, s)
    assert rc == osw.OS_ERR_INVALID_ARG
