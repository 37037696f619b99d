"""A compact set of oracle pins, runnable against any build of the oracle.

``python tests/oracle_pins.py <liboracle.so>`` prints a JSON list of the pins
that fail. ``test_oracle_mutants.py`` runs it on deliberately broken copies of
the oracle (each in a child process, so a broken copy cannot take the test
run down) and expects every copy to fail at least one pin.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import oracle  # noqa: E402
from conftest import read_golden  # noqa: E402
from paper_2206_01784_gb300 import workload  # noqa: E402


def _field(keys, begin, end):
    k = keys.astype(np.uint64)
    w = end - begin
    mask = np.uint64((1 << w) - 1) if w < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    return (k >> np.uint64(begin)) & mask


def _ieee_rank(bits, wide):
    x = bits.view(np.float64 if wide else np.float32)
    return np.lexsort((np.arange(x.size), np.where(np.signbit(x), 0, 1), x))


def _ordered_np(bits, wide):
    """Sign-flip written with numpy; checked against IEEE order in pin_float_np."""
    sign = np.uint64(1 << 63) if wide else np.uint32(1 << 31)
    return np.where(bits & sign, ~bits, bits | sign)


def pin_exclusive_sum():
    g = read_golden("exclusive_sum_section2.txt")
    return oracle.exclusive_sum(g["input"]).tolist() == g["output"]


def pin_flag_scan():
    g = read_golden("flag_scan_section2.txt")
    keys = np.array(g["keys"], np.uint32)
    b = g["digit_bits"][0]
    _, perm = oracle.sort("u32", keys, np.arange(4, dtype=np.uint32), 0, b, b)
    dest = np.empty(4, np.int64)
    dest[perm] = np.arange(4)
    off = oracle.bin_offsets("u32", keys, 0, b, b)[0]
    return all(dest[i] - int(off[0]) == g["offsets"][i] for i in range(4) if g["flags"][i])


def pin_sort_numpy():
    ok = True
    for kt, begin, end in (("u32", 0, 32), ("u32", 13, 31), ("u32", 3, 29), ("u64", 0, 64), ("u64", 5, 50)):
        keys = workload.keys(kt, "and2", 5000, seed=4)
        ko, vo = oracle.sort(kt, keys, workload.iota_u32(keys.size), begin, end)
        perm = np.argsort(_field(keys, begin, end), kind="stable")
        ok &= np.array_equal(vo, perm.astype(np.uint32)) and np.array_equal(ko, keys[perm])
    return bool(ok)


def pin_float():
    ok = True
    for kt, wide in (("f32", False), ("f64", True)):
        bits = workload.keys(kt, "normal", 5000, seed=9)
        ko, vo = oracle.sort(kt, bits, workload.iota_u32(bits.size))
        r = _ieee_rank(bits, wide)
        ok &= np.array_equal(vo, r.astype(np.uint32)) and np.array_equal(ko, bits[r])
    return bool(ok)


def pin_histograms():
    ok = True
    for kt, begin, end in (("u32", 3, 29), ("u64", 0, 64), ("f32", 0, 32)):
        keys = workload.keys("u32" if kt == "f32" else kt, "uniform", 4000, seed=21)
        src = _ordered_np(keys, False) if kt == "f32" else keys
        h = oracle.histograms(kt, keys, begin, end)
        for place in range(h.shape[0]):
            s = begin + 8 * place
            d = _field(src, s, min(s + 8, end)).astype(np.int64)
            ok &= np.array_equal(h[place], np.bincount(d, minlength=256))
    return bool(ok)


def pin_float_np():
    # the numpy sign-flip used above agrees with IEEE order
    bits = workload.keys("f32", "normal", 3000, seed=3)
    return bool(np.array_equal(np.argsort(_ordered_np(bits, False), kind="stable"), _ieee_rank(bits, False)))


def pin_tile_counts():
    keys = workload.keys("u32", "uniform", 3000, seed=13)
    c = oracle.tile_digit_counts("u32", keys, 0, 8, 700)
    return all(np.array_equal(c[t], np.bincount((keys[t * 700:(t + 1) * 700] & 0xFF).astype(np.int64),
                                                minlength=256)) for t in range(c.shape[0]))


def pin_signed():
    bits = workload.keys("i32", "uniform", 4000, seed=17)
    ko, vo = oracle.sort("i32", bits, workload.iota_u32(bits.size))
    perm = np.argsort(bits.view(np.int32), kind="stable")
    return bool(np.array_equal(vo, perm.astype(np.uint32)) and np.array_equal(ko, bits[perm]))


def pin_descending_bruteforce():
    # every array of length <= 4 over 3-bit keys (digit widths 1-3), and
    # seeded length-9 arrays: the stable descending order of Python's sorted
    # (reverse=True keeps equal keys in input order)
    import itertools
    rng = np.random.default_rng(5)
    cases = [np.array(c, np.uint32) for n in range(1, 5) for c in itertools.product(range(8), repeat=n)]
    cases += [rng.integers(0, 8, 9).astype(np.uint32) for _ in range(200)]
    for keys in cases:
        for d in (1, 2, 3):
            _, vo = oracle.sort("u32", keys, np.arange(keys.size, dtype=np.uint32), 0, 3, d, descending=True)
            exp = sorted(range(keys.size), key=lambda i: int(keys[i]), reverse=True)
            if vo.tolist() != exp:
                return False
    return True


def pin_descending_numpy():
    ok = True
    for kt, begin, end in (("u32", 0, 32), ("u32", 3, 29), ("u64", 0, 64), ("u64", 5, 50)):
        keys = workload.keys(kt, "and3", 5000, seed=6)
        ko, vo = oracle.sort(kt, keys, workload.iota_u32(keys.size), begin, end, descending=True)
        f = _field(keys, begin, end)
        perm = np.argsort(f.max() - f, kind="stable")  # descending field, ties in input order
        ok &= np.array_equal(vo, perm.astype(np.uint32)) and np.array_equal(ko, keys[perm])
        h = oracle.histograms(kt, keys, begin, end, descending=True)
        for place in range(h.shape[0]):
            s = begin + 8 * place
            w = min(s + 8, end) - s
            d = ((1 << w) - 1) - _field(keys, s, s + w).astype(np.int64)
            ok &= np.array_equal(h[place], np.bincount(d, minlength=256))
    # float keys: IEEE descending, +0.0 before -0.0, ties in input order
    bits = workload.keys("f32", "normal", 5000, seed=9)
    ko, vo = oracle.sort("f32", bits, workload.iota_u32(bits.size), descending=True)
    x = bits.view(np.float32)
    r = np.lexsort((np.arange(x.size), np.where(np.signbit(x), 1, 0), -x))
    ok &= np.array_equal(vo, r.astype(np.uint32))
    # signed keys
    bits = workload.keys("i64", "uniform", 3000, seed=2)
    _, vo = oracle.sort("i64", bits, workload.iota_u32(bits.size), descending=True)
    ok &= np.array_equal(vo, np.argsort(-bits.view(np.int64).astype(object), kind="stable").astype(np.uint32))
    return bool(ok)


PINS = [pin_signed, pin_exclusive_sum, pin_flag_scan, pin_sort_numpy, pin_float, pin_histograms, pin_float_np,
        pin_tile_counts, pin_descending_bruteforce, pin_descending_numpy]


def failing(lib_path=None):
    if lib_path:
        oracle.use_library(lib_path)
    bad = []
    for pin in PINS:
        try:
            if not pin():
                bad.append(pin.__name__)
        except Exception:  # a broken copy may also raise
            bad.append(pin.__name__)
    return bad


if __name__ == "__main__":
    print(json.dumps(failing(sys.argv[1] if len(sys.argv) > 1 else None)))
