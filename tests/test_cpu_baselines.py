"""The benchmark's CPU comparison rows (oracle/cpu_baselines.cpp: a
multi-threaded LSD radix sort and std::stable_sort) give exactly the
oracle's result, so their timings describe the same sort (no GPU)."""
import numpy as np
import pytest

import oracle
from paper_2206_01784_gb300 import workload


@pytest.mark.parametrize("kt,begin,end", [("u32", 0, 32), ("u32", 3, 29), ("u64", 0, 64), ("u64", 5, 50),
                                          ("f32", 0, 32), ("f64", 0, 64), ("i32", 0, 32), ("i64", 9, 64)])
@pytest.mark.parametrize("pairs", [False, True])
def test_parallel_lsd_and_std_stable_sort_match_oracle(kt, begin, end, pairs):
    for n, dist, threads in ((0, "uniform", 4), (1, "uniform", 4), (5000, "and3", 3), (300_001, "uniform", 7),
                             (300_001, "const", 16)):
        d = "normal" if kt in ("f32", "f64") and dist == "uniform" else dist
        keys = workload.keys(kt, d, n, seed=n + begin)
        vals = workload.iota_u32(n) if pairs else None
        exp = oracle.sort(kt, keys, vals, begin, end)
        for got in (oracle.parallel_sort(kt, keys, vals, begin, end, threads=threads),
                    oracle.std_stable_sort(kt, keys, vals, begin, end)):
            if pairs:
                assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1]), (kt, n)
            else:
                assert np.array_equal(got, exp), (kt, n)


def test_hardware_threads():
    assert oracle.hardware_threads() >= 1
