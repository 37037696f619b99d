"""Parity at the full workload sizes, in the launch configuration bench.py times.

* 2^20 uint32 keys only, uniform, seed 0: bit-exact against the oracle.
* 2^28 uint32 keys + index values, uniform, seed 1: bit-exact against the
  oracle (whole output).
* 2^27 uint64 pairs (seed 8), 2^28 float32 N(0,1) pairs (seed 9) and the
  4096-segment lognormal batch (seed 10): bit-exact against the oracle (whole
  output), and checked by properties that together pin the unique stable
  sort - the output keys are nondecreasing in the sort order, the output
  values are a permutation of the input indices, every output key is the
  input key at its value's index, and equal keys carry increasing indices.
* 2^28 uint32 pairs for the other entropy bands (AND of q = 2..5 words, seeds
  q; all-equal, seed 6; q = 8, 16, seed 7): the same properties. The checks
  run in numpy on the host, independent of the GPU.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2206_01784_gb300 import onesweep as osw  # noqa: E402
from paper_2206_01784_gb300 import workload  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _to_dev(a):
    return torch.from_numpy(a.view(np.int64 if a.dtype.itemsize == 8 else np.int32)).to(_dev())


def _ordered_np(bits):
    """Sort order of float bits (sign-flip), written with numpy for the check."""
    if bits.dtype == np.uint32:
        sign = np.uint32(1 << 31)
    else:
        sign = np.uint64(1 << 63)
    return np.where(bits & sign, ~bits, bits | sign)


def check_stable_sort(keys_in, keys_out, vals_out, order_keys=None):
    """Properties that hold exactly when (keys_out, vals_out) is the stable sort."""
    n = keys_in.size
    ok_in = keys_in if order_keys is None else order_keys(keys_in)
    ok_out = keys_out if order_keys is None else order_keys(keys_out)
    assert np.all(ok_out[1:] >= ok_out[:-1]), "not sorted"
    seen = np.zeros(n, dtype=bool)
    seen[vals_out] = True
    assert seen.all() and vals_out.max(initial=0) < n, "values are not a permutation"
    assert np.array_equal(keys_in[vals_out], keys_out), "keys do not follow their values"
    eq = ok_out[1:] == ok_out[:-1]
    assert np.all(vals_out[1:][eq] > vals_out[:-1][eq]), "not stable"
    del ok_in


def sort_pairs_dev(kt, keys):
    n = keys.size
    k = _to_dev(keys)
    v = _to_dev(workload.iota_u32(n))
    ko, vo = osw.sort_pairs(k, v, key_type=kt)
    torch.cuda.synchronize()
    dt = np.uint64 if keys.dtype == np.uint64 else np.uint32
    return ko.cpu().numpy().view(dt), vo.cpu().numpy().view(np.uint32)


def test_config_1m_u32_keys_exact():
    n = 1 << 20
    keys = workload.keys("u32", "uniform", n, 0)
    out = osw.sort_keys(_to_dev(keys), key_type="u32")
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle.sort("u32", keys))


def test_config_256m_u32_pairs_uniform_exact():
    n = 1 << 28
    keys = workload.keys("u32", "uniform", n, 1)
    ko, vo = sort_pairs_dev("u32", keys)
    ek, ev = oracle.sort("u32", keys, workload.iota_u32(n))
    assert np.array_equal(ko, ek)
    assert np.array_equal(vo, ev)


@pytest.mark.parametrize("dist,seed", [("and2", 2), ("and3", 3), ("and4", 4), ("and5", 5), ("const", 6),
                                       ("and8", 7), ("and16", 7)])
def test_config_256m_u32_pairs_bands(dist, seed):
    n = 1 << 28
    keys = workload.keys("u32", dist, n, seed)
    ko, vo = sort_pairs_dev("u32", keys)
    check_stable_sort(keys, ko, vo)


def test_config_128m_u64_pairs():
    n = 1 << 27
    keys = workload.keys("u64", "uniform", n, 8)
    ko, vo = sort_pairs_dev("u64", keys)
    check_stable_sort(keys, ko, vo)
    ek, ev = oracle.sort("u64", keys, workload.iota_u32(n))
    assert np.array_equal(ko, ek)
    assert np.array_equal(vo, ev)


def test_config_256m_f32_pairs():
    n = 1 << 28
    keys = workload.keys("f32", "normal", n, 9)
    ko, vo = sort_pairs_dev("f32", keys)
    check_stable_sort(keys, ko, vo, order_keys=_ordered_np)
    ek, ev = oracle.sort("f32", keys, workload.iota_u32(n))
    assert np.array_equal(ko, ek.view(np.uint32))
    assert np.array_equal(vo, ev)
    # -0.0 before +0.0 among the zeros
    zeros = ko[(ko & np.uint32(0x7FFFFFFF)) == 0]
    assert zeros.size > 0 and np.all(np.diff((zeros == 0).astype(np.int8)) >= 0)


def test_config_4096_segment_batch():
    sizes = workload.segment_sizes(4096, seed=10)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offs[-1])
    keys = workload.keys("u32", "uniform", n, 10)
    k, v = _to_dev(keys), _to_dev(workload.iota_u32(n))
    ko, vo = osw.sort_batch(k, torch.from_numpy(offs).to(_dev()), v, key_type="u32")
    torch.cuda.synchronize()
    ko, vo = ko.cpu().numpy().view(np.uint32), vo.cpu().numpy().view(np.uint32)
    seg = np.repeat(np.arange(sizes.size), sizes)
    # values stay inside their segment and form a permutation of it
    assert np.all(vo >= offs[:-1][seg]) and np.all(vo < offs[1:][seg])
    seen = np.zeros(n, dtype=bool)
    seen[vo] = True
    assert seen.all()
    assert np.array_equal(keys[vo], ko)
    inside = seg[1:] == seg[:-1]  # neighbours in the same segment
    assert np.all(ko[1:][inside] >= ko[:-1][inside])
    eq = inside & (ko[1:] == ko[:-1])
    assert np.all(vo[1:][eq] > vo[:-1][eq])
    # every segment against the oracle
    ek, ev = oracle.sort_segments("u32", keys, offs.astype(np.uint64), workload.iota_u32(n))
    assert np.array_equal(ko, ek) and np.array_equal(vo, ev)
