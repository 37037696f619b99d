"""The oracle's sort against std::stable_sort (C++ standard library) on the
same keys: for every key type, bit ranges including narrow, odd and empty
ones, and the entropy bands, the oracle's output values (input indices) must
be exactly the permutation std::stable_sort produces on the sorted-on field."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2206_01784_gb300 import workload

HERE = os.path.dirname(os.path.abspath(__file__))
KB = {"u32": 32, "u64": 64, "f32": 32, "f64": 64, "i32": 32, "i64": 64}
KIND = {"u32": 0, "u64": 0, "i32": 1, "i64": 1, "f32": 2, "f64": 2}


@pytest.fixture(scope="module")
def ref(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("stable_sort_ref") / "libstable_sort_ref.so")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", os.path.join(HERE, "stable_sort_ref.cpp"),
                           "-o", out])
    lib = ctypes.CDLL(out)
    vp, sz, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
    for name in ("ref_stable_perm32", "ref_stable_perm64"):
        getattr(lib, name).argtypes = [vp, vp, sz, i32, i32, i32]
        getattr(lib, name).restype = None
    return lib


def _perm(ref, kt, keys, begin, end):
    perm = np.empty(keys.size, np.uint32)
    fn = ref.ref_stable_perm64 if KB[kt] == 64 else ref.ref_stable_perm32
    fn(keys.ctypes.data, perm.ctypes.data, keys.size, begin, end, KIND[kt])
    return perm


@pytest.mark.parametrize("kt", sorted(KB))
@pytest.mark.parametrize("dist", ["uniform", "and3", "const"])
def test_oracle_matches_std_stable_sort(ref, kt, dist):
    n = 20_011
    if kt[0] == "f" and dist == "uniform":
        keys = workload.keys(kt, "normal", n, 77)
    else:
        wide = KB[kt] == 64
        keys = workload.keys("u64" if wide else "u32", dist, n, 77)
    vals = workload.iota_u32(n)
    kb = KB[kt]
    for begin, end in [(0, kb), (0, 8), (3, kb - 5), (kb - 8, kb), (7, 7), (5, 18)]:
        ko, vo = oracle.sort(kt, keys, vals, begin, end)
        perm = _perm(ref, kt, keys, begin, end)
        assert np.array_equal(vo, perm), (kt, dist, begin, end)
        assert np.array_equal(ko, keys[perm])
