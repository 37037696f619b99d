"""Host-buffer entry points (os_sort_keys_host / os_sort_pairs_host) through
the C ABI: keys and values in host memory, page-locked or pageable, sorted
bit-exact against the oracle; two calls in flight on two streams with two
workspaces."""
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


def _keys(kt, n, seed):
    return workload.keys(kt, "normal" if kt in ("f32", "f64") else "and2", n, seed)


def _host_buf(a, pinned):
    """A page-locked host copy of a's bits and its address."""
    assert pinned
    t = torch.from_numpy(a.view(np.int64 if a.dtype.itemsize == 8 else np.int32).copy()).pin_memory()
    return t, t.data_ptr()


def _empty_like(a, pinned):
    if pinned:
        t = torch.empty(a.size, dtype=torch.int64 if a.dtype.itemsize == 8 else torch.int32).pin_memory()
        return t, t.data_ptr()
    e = np.empty_like(a)
    return e, e.ctypes.data


def _as_np(buf, dt):
    return buf.numpy().view(dt) if isinstance(buf, torch.Tensor) else buf.view(dt)


def _run(kt, keys, vals, begin, end, pinned, stream=None):
    dev = _dev()
    n = keys.size
    if pinned:
        hk, pk = _host_buf(keys, True)
    else:
        hk = keys.copy()
        pk = hk.ctypes.data
    hko, pko = _empty_like(keys, pinned)
    pv = pvo = None
    if vals is not None:
        if pinned:
            hv, pv = _host_buf(vals, True)
        else:
            hv = vals.copy()
            pv = hv.ctypes.data
        hvo, pvo = _empty_like(vals, pinned)
    wsb = osw.os_sort_host_workspace_bytes(osw.KEY_TYPES[kt], n, 4 if vals is not None else 0, begin, end)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    s = (stream or torch.cuda.current_stream()).cuda_stream
    if vals is None:
        rc = osw.os_sort_keys_host(osw.KEY_TYPES[kt], pk, pko, n, begin, end, ws.data_ptr(), wsb, s)
    else:
        rc = osw.os_sort_pairs_host(osw.KEY_TYPES[kt], pk, pko, pv, pvo, n, begin, end, ws.data_ptr(), wsb, s)
    assert rc == osw.OS_OK
    assert osw.os_workspace_status(ws.data_ptr(), s) == osw.OS_OK  # waits for the stream
    dt = np.uint64 if KB[kt] == 64 else np.uint32
    ko = _as_np(hko, dt).copy()
    return ko if vals is None else (ko, _as_np(hvo, np.uint32).copy())


@pytest.fixture(params=["engines", "link"])
def copy_mode(request):
    """Both ways the host-memory sorts move data: the copy engines and the
    copy kernels over the host link (page-locked buffers only; others fall
    back to the copy engines)."""
    mode = {"engines": osw.OS_HOST_COPY_ENGINES, "link": osw.OS_HOST_COPY_LINK}[request.param]
    old = osw.os_get_host_copy_mode()
    assert osw.os_set_host_copy_mode(mode) == osw.OS_OK
    yield mode
    osw.os_set_host_copy_mode(old)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("kt,pairs,begin,end", [("u32", True, 0, 32), ("u32", False, 0, 32), ("u64", True, 0, 64),
                                                 ("f32", True, 0, 32), ("i64", True, 3, 64), ("f64", False, 0, 64)])
@pytest.mark.parametrize("n", [300_007, 300_008])
def test_host_sort_exact(kt, pairs, begin, end, pinned, copy_mode, n):
    # 300 008 keys: byte counts that are multiples of 16 (the link copy kernel
    # alone); 300 007: the kernel and a tail through the copy engines
    keys = _keys(kt, n, seed=31)
    vals = workload.iota_u32(n) if pairs else None
    got = _run(kt, keys, vals, begin, end, pinned)
    exp = oracle.sort(kt, keys, vals, begin, end)
    if pairs:
        assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])
    else:
        assert np.array_equal(got, exp)


def test_host_sort_two_streams(copy_mode):
    dev = _dev()
    n = 1 << 20
    ks = [_keys("u32", n, seed=40 + i) for i in range(2)]
    vals = workload.iota_u32(n)
    streams = [torch.cuda.Stream(dev) for _ in range(2)]
    wsb = osw.os_sort_host_workspace_bytes(osw.OS_KEY_U32, n, 4, 0, 32)
    ws = [torch.empty(wsb, dtype=torch.uint8, device=dev) for _ in range(2)]
    hin = [torch.from_numpy(k.view(np.int32).copy()).pin_memory() for k in ks]
    hv = torch.from_numpy(vals.view(np.int32).copy()).pin_memory()
    hko = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in range(2)]
    hvo = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in range(2)]
    for i in range(2):
        rc = osw.os_sort_pairs_host(osw.OS_KEY_U32, hin[i].data_ptr(), hko[i].data_ptr(), hv.data_ptr(),
                                    hvo[i].data_ptr(), n, 0, 32, ws[i].data_ptr(), wsb, streams[i].cuda_stream)
        assert rc == osw.OS_OK
    for i in range(2):
        assert osw.os_workspace_status(ws[i].data_ptr(), streams[i].cuda_stream) == osw.OS_OK
        exp = oracle.sort("u32", ks[i], vals, 0, 32)
        assert np.array_equal(hko[i].numpy().view(np.uint32), exp[0])
        assert np.array_equal(hvo[i].numpy().view(np.uint32), exp[1])


def test_host_sort_empty_and_copy():
    # n = 0 is a no-op; an empty bit range copies the input through
    _dev()
    assert osw.os_sort_keys_host(osw.OS_KEY_U32, None, None, 0, 0, 32, None, 0, 0) == osw.OS_OK
    keys = _keys("u32", 5000, seed=3)
    got = _run("u32", keys, workload.iota_u32(5000), 7, 7, True)
    assert np.array_equal(got[0], keys) and np.array_equal(got[1], workload.iota_u32(5000))


@pytest.mark.parametrize("kt,pairs", [("u32", True), ("f32", False), ("u64", True), ("i32", True)])
def test_binding_sort_host_numpy(kt, pairs):
    # the binding's host-array helper: numpy in, numpy out, one host-buffer call
    _dev()
    n = 123_457
    keys = _keys(kt, n, seed=55)
    vals = workload.iota_u32(n) if pairs else None
    got = osw.sort_host(keys, vals, key_type=kt)
    exp = oracle.sort(kt, keys, vals)
    if pairs:
        assert np.array_equal(got[0].view(exp[0].dtype), exp[0]) and np.array_equal(got[1].view(np.uint32), exp[1])
    else:
        assert np.array_equal(got.view(exp.dtype), exp)


@pytest.mark.parametrize("offset,n", [(0, 4100), (0, 4099), (0, 3), (1, 4100), (4, 4100), (3, 70001)])
def test_host_link_mode_unaligned_and_odd_sizes(offset, n, copy_mode):
    # in the link mode, host buffers that start off a 16-byte boundary (offsets
    # 1 and 3 words) take the copy engines; aligned ones (offsets 0 and 4
    # words) the copy kernel, plus the copy engines for a tail of fewer than
    # 16 bytes (n = 4099) or for a buffer of fewer than 16 bytes (n = 3):
    # every case bit-exact
    dev = _dev()
    keys = _keys("u32", n, seed=61 + offset + n)
    vals = workload.iota_u32(n)
    pad = torch.empty(n + 8, dtype=torch.int32).pin_memory()
    padv = torch.empty(n + 8, dtype=torch.int32).pin_memory()
    hk, hv = pad[offset:offset + n], padv[offset:offset + n]
    hk.copy_(torch.from_numpy(keys.view(np.int32)))
    hv.copy_(torch.from_numpy(vals.view(np.int32)))
    hko = torch.empty(n + 8, dtype=torch.int32).pin_memory()[offset:offset + n]
    hvo = torch.empty(n + 8, dtype=torch.int32).pin_memory()[offset:offset + n]
    wsb = osw.os_sort_host_workspace_bytes(osw.OS_KEY_U32, n, 4, 0, 32)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream().cuda_stream
    rc = osw.os_sort_pairs_host(osw.OS_KEY_U32, hk.data_ptr(), hko.data_ptr(), hv.data_ptr(), hvo.data_ptr(), n, 0,
                                32, ws.data_ptr(), wsb, s)
    assert rc == osw.OS_OK
    assert osw.os_workspace_status(ws.data_ptr(), s) == osw.OS_OK
    exp = oracle.sort("u32", keys, vals, 0, 32)
    assert np.array_equal(hko.numpy().view(np.uint32), exp[0])
    assert np.array_equal(hvo.numpy().view(np.uint32), exp[1])
