"""Concurrent callers: several host threads, each on its own stream with its
own workspace and its own binning variant (os_sort_pairs_ex /
os_sort_keys_ex), sort at the same time; every result is bit-exact against
the CPU oracle. The library keeps no per-call state outside the call's
arguments, so nothing is shared between the threads but the device."""
import threading

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


def _worker(tid, cfg, rounds, results, errors):
    try:
        dev = _dev()
        torch.cuda.set_device(dev)
        stream = torch.cuda.Stream(dev)
        n = 300_000 + 70_001 * tid
        pairs = tid % 2 == 0
        ws = osw.workspace(osw.OS_KEY_U32, n, 4 if pairs else 0, 0, 32, dev)
        for r in range(rounds):
            keys = workload.keys("u32", ("uniform", "and3")[r % 2], n, seed=1000 * tid + r)
            with torch.cuda.stream(stream):
                k = torch.from_numpy(keys.view(np.int32).copy()).to(dev, non_blocking=False)
                ko = torch.empty_like(k)
                s = stream.cuda_stream
                if pairs:
                    vals = workload.iota_u32(n)
                    v = torch.from_numpy(vals.view(np.int32).copy()).to(dev)
                    vo = torch.empty_like(v)
                    rc = osw.os_sort_pairs_ex(osw.OS_KEY_U32, k.data_ptr(), ko.data_ptr(), v.data_ptr(), vo.data_ptr(),
                                              n, 0, 32, ws.data_ptr(), ws.numel(), s, tile_config=cfg)
                else:
                    rc = osw.os_sort_keys_ex(osw.OS_KEY_U32, k.data_ptr(), ko.data_ptr(), n, 0, 32, ws.data_ptr(),
                                             ws.numel(), s, tile_config=cfg)
                assert rc == osw.OS_OK, osw.os_status_string(rc)
                assert osw.os_workspace_status(ws.data_ptr(), s) == osw.OS_OK
                got_k = ko.cpu().numpy().view(np.uint32)
                if pairs:
                    ek, ev = oracle.sort("u32", keys, vals)
                    ok = np.array_equal(got_k, ek) and np.array_equal(vo.cpu().numpy().view(np.uint32), ev)
                else:
                    ok = np.array_equal(got_k, oracle.sort("u32", keys))
            results.append((tid, cfg, r, ok))
    except Exception as e:  # reported by the main thread
        errors.append((tid, repr(e)))


def test_threads_with_their_own_streams_and_variants():
    _dev()
    osw.load()
    n_cfg = osw.os_num_tile_configs()
    # one thread per variant family: one-block-per-tile geometries 0-2 and the
    # persistent kernel, with different ranking methods
    cfgs = [4, 3 + 4, 1, 2 + 8]
    assert all(c < n_cfg for c in cfgs)
    results, errors = [], []
    threads = [threading.Thread(target=_worker, args=(i, c, 4, results, errors)) for i, c in enumerate(cfgs)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert not errors, errors
    assert len(results) == 4 * len(cfgs)
    assert all(ok for *_, ok in results), [r for r in results if not r[-1]]


def test_options_validation():
    _dev()
    n = 1000
    k = torch.zeros(n, dtype=torch.int32, device=_dev())
    ko = torch.empty_like(k)
    ws = osw.workspace(osw.OS_KEY_U32, n, 0, 0, 32, k.device)
    s = torch.cuda.current_stream().cuda_stream
    bad = osw.os_num_tile_configs()
    rc = osw.os_sort_keys_ex(osw.OS_KEY_U32, k.data_ptr(), ko.data_ptr(), n, 0, 32, ws.data_ptr(), ws.numel(), s,
                             tile_config=bad)
    assert rc == osw.OS_ERR_INVALID_ARG
    rc = osw.os_sort_keys_ex(osw.OS_KEY_U32, k.data_ptr(), ko.data_ptr(), n, 0, 32, ws.data_ptr(), ws.numel(), s,
                             tile_config=-1)
    assert rc == osw.OS_OK
