"""Pins of the CPU oracle against what the paper and plain mathematics fix (no GPU).

Each test checks the oracle against something other than itself: the paper's
worked examples (golden fixtures), Python's and numpy's stable sorts, IEEE-754
ordering, exhaustive enumeration of tiny inputs, and invariants.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import lookback_sim
from paper_2206_01784_gb300 import workload
from conftest import read_golden

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _field_np(keys, begin, end):
    keys = np.asarray(keys)
    width = end - begin
    if width == 0:
        return np.zeros(keys.shape, np.uint64)
    k = keys.astype(np.uint64)
    mask = np.uint64((1 << width) - 1) if width < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    return (k >> np.uint64(begin)) & mask


def _float_order_bits_np(bits, wide):
    """IEEE ordering written with numpy comparisons: rank of each float value.

    Used only to check the oracle's transform; independent of its code."""
    if wide:
        x = bits.view(np.float64)
    else:
        x = bits.view(np.float32)
    neg_zero_first = np.where(np.signbit(x), 0, 1)
    return np.lexsort((np.arange(x.size), neg_zero_first, x))


# ---------------------------------------------------------------- Section 2 examples

def test_exclusive_sum_worked_example():
    g = read_golden("exclusive_sum_section2.txt")
    out = oracle.exclusive_sum(g["input"])
    assert out.tolist() == g["output"]


def test_exclusive_sum_definition_random():
    rng = np.random.default_rng(5)
    a = rng.integers(0, 1000, 300).astype(np.uint64)
    out = oracle.exclusive_sum(a)
    # each output is the sum of all inputs strictly before it
    for i in (0, 1, 2, 17, 299):
        assert int(out[i]) == int(a[:i].sum())


def test_flag_scan_worked_example():
    g = read_golden("flag_scan_section2.txt")
    keys = np.array(g["keys"], np.uint32)
    bits = g["digit_bits"][0]
    digit = g["digit"][0]
    idx = np.arange(keys.size, dtype=np.uint32)
    _, perm = oracle.sort("u32", keys, idx, begin_bit=0, end_bit=bits, radix_bits=bits)
    dest = np.empty(keys.size, np.int64)
    dest[perm] = np.arange(keys.size)
    offs = oracle.bin_offsets("u32", keys, 0, bits, bits)[0]
    flags = [(int(k) & ((1 << bits) - 1)) == digit for k in keys]
    assert [int(f) for f in flags] == g["flags"]
    expected_scan = g["offsets"]
    for i, f in enumerate(flags):
        if f:
            assert dest[i] - int(offs[digit]) == expected_scan[i]


def test_bin_relative_offsets_are_flag_prefix_sums():
    # Section 2: for every digit, the scatter offset inside its bin is the
    # exclusive prefix sum of that digit's flags.
    rng = np.random.default_rng(11)
    keys = rng.integers(0, 1 << 32, 500, dtype=np.uint64).astype(np.uint32)
    idx = np.arange(keys.size, dtype=np.uint32)
    _, perm = oracle.sort("u32", keys, idx, begin_bit=8, end_bit=16)
    dest = np.empty(keys.size, np.int64)
    dest[perm] = np.arange(keys.size)
    digits = (keys >> 8) & 0xFF
    offs = oracle.bin_offsets("u32", keys, 8, 16)[0]
    for d in range(256):
        flags = (digits == d).astype(np.int64)
        scan = np.cumsum(flags) - flags
        sel = flags.astype(bool)
        assert np.array_equal(dest[sel] - int(offs[d]), scan[sel])


# ---------------------------------------------------------------- Figure 7

def test_lookback_figure7_every_interleaving():
    g = read_golden("lookback_figure7.txt")
    finals, stuck = lookback_sim.explore(g["local"])
    assert not stuck
    assert finals == {tuple((lookback_sim.G, v) for v in g["inclusive"])}


def test_lookback_figure7_timeline():
    # Replays the states the text describes for Figure 7 (b) through (f).
    g = read_golden("lookback_figure7.txt")
    N, L, G = lookback_sim.N, lookback_sim.L, lookback_sim.G
    c = g["local"]
    # (b): every tile but #2 has published its local count
    sched_b = [0, 1, 3, 4]
    # (c): #2 publishes its count; #0 and #1 finish; #3 adds #2's count and #4
    # adds the counts of #3 and #2
    sched_c = [2, 0, 1, 1, 3, 4, 4]
    # (d): #2 and #3 read #1's G (26) and finish
    sched_d = [2, 2, 3, 3]
    # (e): #4 reads the inclusive count 26 (held by tile #1's counter) and finishes
    sched_e = [4, 4]
    h = lookback_sim.run_schedule(c, sched_b + sched_c + sched_d + sched_e)
    b = h[len(sched_b) - 1]
    assert b == ((L, 11), (L, 15), (N, 0), (L, 10), (L, 8))
    cc = h[len(sched_b) + len(sched_c) - 1]
    assert cc[0] == (G, 11) and cc[1] == (G, 26) and cc[3][0] == L and cc[4][0] == L
    d = h[len(sched_b) + len(sched_c) + len(sched_d) - 1]
    assert d[2] == (G, 35) and d[3] == (G, 45) and d[4][0] == L
    e = h[-1]
    assert e == tuple((G, v) for v in g["inclusive"])


def test_lookback_random_counts_all_interleavings():
    rng = np.random.default_rng(3)
    for g in (1, 2, 3, 4):
        counts = [int(x) for x in rng.integers(0, 20, g)]
        finals, stuck = lookback_sim.explore(counts)
        assert not stuck
        assert finals == {tuple((lookback_sim.G, int(v)) for v in np.cumsum(counts))}


# ---------------------------------------------------------------- histograms

@pytest.mark.parametrize("kt,begin,end", [("u32", 0, 32), ("u32", 3, 29), ("u64", 0, 64),
                                          ("u64", 5, 50), ("f32", 0, 32)])
def test_histograms_direct_count(kt, begin, end):
    n = 20000
    keys = workload.keys(kt if kt != "f32" else "u32", "uniform", n, seed=21)
    h = oracle.histograms(kt, keys, begin, end)
    p = oracle.num_places(begin, end)
    assert h.shape == (p, 256)
    assert np.all(h.sum(axis=1) == n)
    if kt == "f32":
        return
    for place in range(p):
        shift = begin + 8 * place
        width = min(8, end - shift)
        d = _field_np(keys, shift, shift + width)
        ref = np.bincount(d.astype(np.int64), minlength=256)
        assert np.array_equal(h[place], ref)


def test_num_places():
    assert oracle.num_places(0, 32) == 4
    assert oracle.num_places(0, 64) == 8
    assert oracle.num_places(0, 32, 7) == 5  # d=7 (the older CUB radix, Section 3)
    assert oracle.num_places(3, 29) == 4
    assert oracle.num_places(5, 5) == 0


# ---------------------------------------------------------------- full sort

def test_sort_exhaustive_tiny():
    # every array of length <= 6 over 3-bit keys, digit widths 1..3, against a
    # stable numpy argsort of each row (and Python's sorted on a subset)
    for length in range(0, 7):
        rows = np.array(list(itertools.product(range(8), repeat=length)), dtype=np.uint32)
        m = rows.shape[0]
        rows = rows.reshape(m, length)
        flat = rows.reshape(-1)
        offsets = np.arange(m + 1, dtype=np.uint64) * length
        idx = np.tile(np.arange(length, dtype=np.uint32), m)
        expect = np.argsort(rows, axis=1, kind="stable").astype(np.uint32)
        for d in (1, 2, 3):
            ko, vo = oracle.sort_segments("u32", flat, offsets, idx, 0, 3, d)
            assert np.array_equal(vo.reshape(m, length), expect.reshape(m, length))
            assert np.array_equal(ko.reshape(m, length), np.take_along_axis(rows, expect.astype(np.int64), 1))
        if length <= 4:
            for r in rows[:: max(1, m // 200)]:
                ref = sorted(range(length), key=lambda i: (int(r[i]), i))
                _, v = oracle.sort("u32", r, np.arange(length, dtype=np.uint32), 0, 3, 2)
                assert v.tolist() == ref


@pytest.mark.parametrize("kt", ["u32", "u64"])
@pytest.mark.parametrize("begin,end", [(0, None), (0, 8), (4, 20), (7, 7), (13, 31)])
def test_sort_vs_numpy_stable(kt, begin, end):
    kb = 64 if kt == "u64" else 32
    end = kb if end is None else end
    n = 30000
    keys = workload.keys(kt, "and2", n, seed=4)
    vals = workload.iota_u32(n)
    ko, vo = oracle.sort(kt, keys, vals, begin, end)
    perm = np.argsort(_field_np(keys, begin, end), kind="stable")
    assert np.array_equal(vo, perm.astype(np.uint32))
    assert np.array_equal(ko, keys[perm])


@pytest.mark.parametrize("kt", ["f32", "f64"])
def test_float_sort_matches_ieee_order(kt):
    n = 40000
    bits = workload.keys(kt, "normal", n, seed=9)
    wide = kt == "f64"
    specials32 = [0x7F800000, 0xFF800000, 0x00000001, 0x80000001, 0x7F7FFFFF, 0xFF7FFFFF,
                  0x80000000, 0x00000000, 0x3F800000, 0xBF800000]
    specials64 = [0x7FF0000000000000, 0xFFF0000000000000, 1, 0x8000000000000001,
                  0x7FEFFFFFFFFFFFFF, 0xFFEFFFFFFFFFFFFF, 0x8000000000000000, 0, 0x3FF0000000000000,
                  0xBFF0000000000000]
    sp = np.array(specials64 if wide else specials32, dtype=bits.dtype)
    bits = np.concatenate([bits, sp, sp])
    vals = np.arange(bits.size, dtype=np.uint32)
    ko, vo = oracle.sort(kt, bits, vals)
    expect = _float_order_bits_np(bits, wide)
    assert np.array_equal(vo, expect.astype(np.uint32))
    assert np.array_equal(ko, bits[expect])


def test_float_transform_bijective_and_monotone():
    rng = np.random.default_rng(8)
    pats = rng.integers(0, 1 << 32, 2000, dtype=np.uint64)
    for b in pats:
        u = oracle.to_ordered("f32", int(b))
        assert oracle.from_ordered("f32", u) == int(b)
    # -0.0 maps just below +0.0; NaNs sit at the ends
    assert oracle.to_ordered("f32", 0x80000000) + 1 == oracle.to_ordered("f32", 0x00000000)
    assert oracle.to_ordered("f32", 0xFFC00000) < oracle.to_ordered("f32", 0xFF800000)  # -NaN < -inf
    assert oracle.to_ordered("f32", 0x7FC00000) > oracle.to_ordered("f32", 0x7F800000)  # +NaN > +inf
    assert oracle.to_ordered("f64", 0x8000000000000000) + 1 == oracle.to_ordered("f64", 0)
    # unsigned keys are left alone
    assert oracle.to_ordered("u32", 0xDEADBEEF) == 0xDEADBEEF


@pytest.mark.parametrize("dist", ["uniform", "and3", "and5", "and16", "const"])
def test_sort_invariants(dist):
    n = 50000
    keys = workload.keys("u32", dist, n, seed=1)
    vals = workload.iota_u32(n)
    ko, vo = oracle.sort("u32", keys, vals)
    assert np.all(ko[1:] >= ko[:-1])                       # sorted
    assert np.array_equal(np.sort(vo), vals)               # permutation
    assert np.array_equal(ko, keys[vo])                    # keys follow their payload
    eq = ko[1:] == ko[:-1]
    assert np.all(vo[1:][eq] > vo[:-1][eq])                # stable


def test_sort_passes_is_prefix_of_places():
    n = 5000
    keys = workload.keys("u32", "uniform", n, seed=2)
    one = oracle.sort("u32", keys, passes=1)
    assert np.array_equal(one, keys[np.argsort(keys & 0xFF, kind="stable")])
    two = oracle.sort("u32", keys, passes=2)
    assert np.array_equal(two, keys[np.argsort(keys & 0xFFFF, kind="stable")])


def test_sort_keys_only_equals_pairs_keys():
    keys = workload.keys("u64", "and2", 7000, seed=6)
    a = oracle.sort("u64", keys)
    b, _ = oracle.sort("u64", keys, workload.iota_u32(keys.size))
    assert np.array_equal(a, b)


def test_segments_are_independent():
    sizes = [0, 5, 300, 1, 0, 1000]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    keys = workload.keys("u32", "and2", int(off[-1]), seed=12)
    ko = oracle.sort_segments("u32", keys, off)
    for s in range(len(sizes)):
        lo, hi = int(off[s]), int(off[s + 1])
        assert np.array_equal(ko[lo:hi], np.sort(keys[lo:hi], kind="stable"))


def test_tile_digit_counts_prefix():
    n = 10000
    keys = workload.keys("u32", "uniform", n, seed=13)
    c = oracle.tile_digit_counts("u32", keys, 0, 8, 777)
    assert c.shape == ((n + 776) // 777, 256)
    assert np.array_equal(c.sum(axis=0), oracle.histograms("u32", keys, 0, 8)[0])
    t = 5
    ref = np.bincount((keys[t * 777:(t + 1) * 777] & 0xFF).astype(np.int64), minlength=256)
    assert np.array_equal(c[t], ref)


# ---------------------------------------------------------------- generator (Table 1)

def test_entropy_closed_form_matches_table1():
    g = read_golden("entropy_table1.txt")
    for q, h in g["rows"]:
        assert abs(workload.entropy_per_bit(int(q)) - h) < 1e-6


def test_generator_entropy_bands_match_table1():
    g = read_golden("entropy_table1.txt")
    n = 1 << 21
    for q, h in g["rows"]:
        keys = workload.u32_and(n, seed=100 + int(q), q=int(q))
        ones = int(np.unpackbits(keys.view(np.uint8)).sum())
        p = ones / (32.0 * n)
        est = 0.0 if p in (0.0, 1.0) else -(p * np.log2(p) + (1 - p) * np.log2(1 - p))
        assert abs(est - h) <= max(1e-3, 0.1 * h), (q, est, h)


@pytest.mark.parametrize("kt,np_t", [("i32", np.int32), ("i64", np.int64)])
def test_signed_sort_matches_numpy_signed_order(kt, np_t):
    n = 30000
    bits = workload.keys(kt, "uniform", n, seed=17)
    ext = np.array([0, 1, -1, np.iinfo(np_t).min, np.iinfo(np_t).max], dtype=np_t).view(bits.dtype)
    bits = np.concatenate([bits, ext, ext])
    vals = np.arange(bits.size, dtype=np.uint32)
    ko, vo = oracle.sort(kt, bits, vals)
    perm = np.argsort(bits.view(np_t), kind="stable")
    assert np.array_equal(vo, perm.astype(np.uint32))
    assert np.array_equal(ko, bits[perm])
    # a range below the sign bit sorts the raw sub-field
    kb = 64 if kt == "i64" else 32
    ko2, vo2 = oracle.sort(kt, bits, vals, 4, kb - 4)
    assert np.array_equal(vo2, np.argsort(_field_np(bits, 4, kb - 4), kind="stable").astype(np.uint32))
