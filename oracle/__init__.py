"""CPU oracle for Onesweep LSD radix sorting (arXiv 2206.01784).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package. The product path never
calls it and shares no code with it.

The arithmetic lives in ``onesweep_oracle.c`` (plain C, one key at a time,
64-bit counters), compiled by gcc into ``liboracle.so`` beside this file; this
module only marshals numpy arrays. ``lookback_sim`` holds a pure-Python model
of the chained-scan status-counter protocol for small cases.

``cpu_baselines.cpp`` (``libcpu_baselines.so``) is not the oracle: it holds
the benchmark's CPU comparison rows, a multi-threaded LSD radix sort and
std::stable_sort, each checked bit for bit against the oracle
(``tests/test_cpu_baselines.py``); ``parallel_sort`` and ``std_stable_sort``
call them.

Pins (checked in ``tests/test_oracle.py`` without a GPU):
  * exclusive sum: the paper's worked example (Section 2), golden fixture;
  * one binning pass: the paper's flag prefix-sum example (Section 2);
  * chained scan: Figure 7's values under every interleaving (Section 3);
  * full sort: against Python's stable ``sorted`` on tiny exhaustive inputs and
    numpy's stable argsort on random inputs; sortedness, permutation and
    stability invariants; per-place histograms summing to n; the float
    transform against IEEE-754 ordering.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "onesweep_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

KEY_TYPES = {"u32": 0, "u64": 1, "f32": 2, "f64": 3, "i32": 4, "i64": 5}
RADIX_BITS = 8


_CPB_SRC = os.path.join(_HERE, "cpu_baselines.cpp")
_CPB_PATH = os.path.join(_HERE, "libcpu_baselines.so")
_cpb = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no CUDA involved), and the CPU baselines
    with g++."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    if force or not os.path.exists(_CPB_PATH) or os.path.getmtime(_CPB_PATH) < os.path.getmtime(_CPB_SRC):
        tmp = _CPB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O3", "-std=c++17", "-pthread", "-fPIC", "-shared", _CPB_SRC, "-o", tmp])
        os.replace(tmp, _CPB_PATH)
    return _LIB_PATH


def _load_baselines():
    global _cpb
    if _cpb is None:
        build()
        lib = ctypes.CDLL(_CPB_PATH)
        i32, u64, vp = ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p
        lib.cpb_parallel_lsd.restype = i32
        lib.cpb_parallel_lsd.argtypes = [i32, vp, vp, u64, i32, i32, i32, vp, vp]
        lib.cpb_std_stable_sort.restype = i32
        lib.cpb_std_stable_sort.argtypes = [i32, vp, vp, u64, i32, i32, vp, vp]
        lib.cpb_hardware_threads.restype = i32
        lib.cpb_hardware_threads.argtypes = []
        _cpb = lib
    return _cpb


def hardware_threads() -> int:
    """Host threads the multi-threaded baseline uses by default."""
    return int(_load_baselines().cpb_hardware_threads())


def _baseline_call(fn, key_type, keys, vals, begin_bit, end_bit, *extra):
    end_bit = key_bits(key_type) if end_bit is None else end_bit
    k = _keys(key_type, keys)
    ko = np.empty_like(k)
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32)
    vo = None if v is None else np.empty_like(v)
    args = [_kt(key_type), _ptr(k), _ptr(v), k.size, begin_bit, end_bit, *extra, _ptr(ko), _ptr(vo)]
    if fn(*args) != 0:
        raise ValueError("bad arguments")
    return ko if v is None else (ko, vo)


def parallel_sort(key_type: str, keys, vals=None, begin_bit: int = 0, end_bit: int | None = None,
                  threads: int | None = None):
    """The multi-threaded CPU LSD baseline (stable ascending; not the oracle)."""
    lib = _load_baselines()
    return _baseline_call(lib.cpb_parallel_lsd, key_type, keys, vals, begin_bit, end_bit,
                          threads if threads else hardware_threads())


def std_stable_sort(key_type: str, keys, vals=None, begin_bit: int = 0, end_bit: int | None = None):
    """std::stable_sort of the ordered field on one thread (not the oracle)."""
    return _baseline_call(_load_baselines().cpb_std_stable_sort, key_type, keys, vals, begin_bit, end_bit)


def use_library(path: str) -> None:
    """Load the oracle from another build of ``onesweep_oracle.c`` (tests only:
    used to check that the pins reject deliberately broken copies)."""
    global _lib
    _lib = None
    _load(path)


def _load(path: str | None = None):
    global _lib
    if _lib is None:
        if path is None:
            build()
        lib = ctypes.CDLL(path or _LIB_PATH)
        i32, u64, i64, vp = ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p
        lib.orc_key_bits.restype = i32
        lib.orc_key_bits.argtypes = [i32]
        lib.orc_to_ordered.restype = u64
        lib.orc_to_ordered.argtypes = [i32, u64]
        lib.orc_from_ordered.restype = u64
        lib.orc_from_ordered.argtypes = [i32, u64]
        lib.orc_num_places.restype = i32
        lib.orc_num_places.argtypes = [i32, i32, i32]
        lib.orc_exclusive_sum.restype = None
        lib.orc_exclusive_sum.argtypes = [vp, i64, vp]
        lib.orc_histograms.restype = None
        lib.orc_histograms.argtypes = [i32, vp, u64, i32, i32, i32, vp]
        lib.orc_bin_offsets.restype = None
        lib.orc_bin_offsets.argtypes = [i32, vp, u64, i32, i32, i32, vp]
        lib.orc_sort.restype = i32
        lib.orc_sort.argtypes = [i32, vp, vp, u64, i32, i32, i32, vp, vp]
        lib.orc_sort_passes.restype = i32
        lib.orc_sort_passes.argtypes = [i32, vp, vp, u64, i32, i32, i32, i32, vp, vp]
        lib.orc_sort_segments.restype = i32
        lib.orc_sort_segments.argtypes = [i32, vp, vp, vp, i64, i32, i32, i32, vp, vp]
        lib.orc_histograms_ex.restype = None
        lib.orc_histograms_ex.argtypes = [i32, vp, u64, i32, i32, i32, i32, vp]
        lib.orc_bin_offsets_ex.restype = None
        lib.orc_bin_offsets_ex.argtypes = [i32, vp, u64, i32, i32, i32, i32, vp]
        lib.orc_sort_ex.restype = i32
        lib.orc_sort_ex.argtypes = [i32, vp, vp, u64, i32, i32, i32, i32, vp, vp]
        lib.orc_sort_segments_ex.restype = i32
        lib.orc_sort_segments_ex.argtypes = [i32, vp, vp, vp, i64, i32, i32, i32, i32, vp, vp]
        lib.orc_tile_digit_counts.restype = i32
        lib.orc_tile_digit_counts.argtypes = [i32, vp, u64, i32, i32, u64, vp]
        _lib = lib
    return _lib


def _kt(key_type: str) -> int:
    return KEY_TYPES[key_type]


def _key_dtype(key_type: str):
    return np.uint64 if key_type in ("u64", "f64", "i64") else np.uint32


def _keys(key_type: str, keys) -> np.ndarray:
    return np.ascontiguousarray(keys, dtype=_key_dtype(key_type))


def _ptr(a) -> int | None:
    return None if a is None else a.ctypes.data


def key_bits(key_type: str) -> int:
    return 64 if key_type in ("u64", "f64", "i64") else 32


def to_ordered(key_type: str, bits: int) -> int:
    return int(_load().orc_to_ordered(_kt(key_type), int(bits)))


def from_ordered(key_type: str, u: int) -> int:
    return int(_load().orc_from_ordered(_kt(key_type), int(u)))


def num_places(begin_bit: int, end_bit: int, radix_bits: int = RADIX_BITS) -> int:
    return int(_load().orc_num_places(begin_bit, end_bit, radix_bits))


def exclusive_sum(counts) -> np.ndarray:
    a = np.ascontiguousarray(counts, dtype=np.uint64)
    out = np.empty_like(a)
    _load().orc_exclusive_sum(_ptr(a), a.size, _ptr(out))
    return out


def histograms(key_type: str, keys, begin_bit: int = 0, end_bit: int | None = None,
               radix_bits: int = RADIX_BITS, descending: bool = False) -> np.ndarray:
    """[p, 2^radix_bits] digit counts of every place (uint64); for a descending
    sort, of the complemented digits the passes bin by."""
    end_bit = key_bits(key_type) if end_bit is None else end_bit
    k = _keys(key_type, keys)
    p = num_places(begin_bit, end_bit, radix_bits)
    out = np.zeros((max(p, 1), 1 << radix_bits), np.uint64)
    _load().orc_histograms_ex(_kt(key_type), _ptr(k), k.size, begin_bit, end_bit, radix_bits, int(descending),
                              _ptr(out))
    return out[:p]


def bin_offsets(key_type: str, keys, begin_bit: int = 0, end_bit: int | None = None,
                radix_bits: int = RADIX_BITS, descending: bool = False) -> np.ndarray:
    """[p, 2^radix_bits] global bin offsets (exclusive sums of the histograms)."""
    end_bit = key_bits(key_type) if end_bit is None else end_bit
    k = _keys(key_type, keys)
    p = num_places(begin_bit, end_bit, radix_bits)
    out = np.zeros((max(p, 1), 1 << radix_bits), np.uint64)
    _load().orc_bin_offsets_ex(_kt(key_type), _ptr(k), k.size, begin_bit, end_bit, radix_bits, int(descending),
                               _ptr(out))
    return out[:p]


def sort(key_type: str, keys, vals=None, begin_bit: int = 0, end_bit: int | None = None,
         radix_bits: int = RADIX_BITS, passes: int | None = None, descending: bool = False):
    """Stable ascending (or stable descending) LSD sort. Returns keys, or
    (keys, vals) when vals is given.

    ``passes`` stops after that many binning passes (default: all p; an
    ascending sort only)."""
    end_bit = key_bits(key_type) if end_bit is None else end_bit
    k = _keys(key_type, keys)
    ko = np.empty_like(k)
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32)
    vo = None if v is None else np.empty_like(v)
    lib = _load()
    if passes is None:
        rc = lib.orc_sort_ex(_kt(key_type), _ptr(k), _ptr(v), k.size, begin_bit, end_bit, radix_bits,
                             int(descending), _ptr(ko), _ptr(vo))
    elif descending:
        raise ValueError("passes applies to ascending sorts")
    else:
        rc = lib.orc_sort_passes(_kt(key_type), _ptr(k), _ptr(v), k.size, begin_bit, end_bit, radix_bits,
                                 passes, _ptr(ko), _ptr(vo))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return ko if v is None else (ko, vo)


def sort_segments(key_type: str, keys, offsets, vals=None, begin_bit: int = 0, end_bit: int | None = None,
                  radix_bits: int = RADIX_BITS, descending: bool = False):
    """Each segment [offsets[s], offsets[s+1]) sorted on its own."""
    end_bit = key_bits(key_type) if end_bit is None else end_bit
    k = _keys(key_type, keys)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    ko = np.empty_like(k)
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32)
    vo = None if v is None else np.empty_like(v)
    rc = _load().orc_sort_segments_ex(_kt(key_type), _ptr(k), _ptr(v), _ptr(off), off.size - 1, begin_bit,
                                      end_bit, radix_bits, int(descending), _ptr(ko), _ptr(vo))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return ko if v is None else (ko, vo)


def tile_digit_counts(key_type: str, keys, shift: int, width: int, tile: int) -> np.ndarray:
    """[tiles, 2^width] digit counts of each tile of ``tile`` consecutive keys."""
    k = _keys(key_type, keys)
    tiles = (k.size + tile - 1) // tile
    out = np.zeros((max(tiles, 1), 1 << width), np.uint64)
    rc = _load().orc_tile_digit_counts(_kt(key_type), _ptr(k), k.size, shift, width, tile, _ptr(out))
    if rc != 0:
        raise ValueError("bad tile size")
    return out[:tiles]
