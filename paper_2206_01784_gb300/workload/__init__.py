"""Seeded synthetic inputs for the Onesweep radix sort (arXiv 2206.01784, Section 4).

This module draws inputs only; it holds none of the sort's arithmetic. Both the
CUDA path and the CPU oracle are fed from it. The generator itself is C
(``gen.c``, SplitMix64, counter-based) compiled into ``libworkload.so`` beside
this file.

Workloads (the paper's Section 4 shapes, made synthetic and seeded):

* ``uniform`` - uniform random words (entropy band q=1).
* ``andK``    - bitwise AND of K uniform words (Thearling-Smith bands,
  Table 1: each bit is set with probability 2^-K).
* ``const``   - all-equal keys.
* ``normal``  - float keys N(0,1) with 0.5% -0.0, 0.5% +0.0 and 1% duplicates.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libworkload.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libworkload.so (gcc, OpenMP)."""
    import subprocess

    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", src, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            build()
        lib = ctypes.CDLL(_LIB_PATH)
        u64, i32, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
        lib.wl_splitmix64.restype = u64
        lib.wl_splitmix64.argtypes = [u64, u64]
        lib.wl_stream_seed.restype = u64
        lib.wl_stream_seed.argtypes = [u64, u64]
        for name in ("wl_u32_and", "wl_u64_and"):
            getattr(lib, name).argtypes = [vp, u64, u64, i32]
        for name in ("wl_u32_const", "wl_u64_const", "wl_f32_normal", "wl_f64_normal"):
            getattr(lib, name).argtypes = [vp, u64, u64]
        lib.wl_iota_u32.argtypes = [vp, u64]
        lib.wl_uniform01.argtypes = [vp, u64, u64, u64]
        lib.wl_normal.argtypes = [vp, u64, u64, u64]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def splitmix64(seed: int, i: int) -> int:
    """Output number i (0-based) of SplitMix64 seeded with ``seed``."""
    return int(_load().wl_splitmix64(seed & (2**64 - 1), i))


def u32_and(n: int, seed: int, q: int, out: np.ndarray | None = None) -> np.ndarray:
    out = np.empty(n, np.uint32) if out is None else out
    _load().wl_u32_and(_ptr(out), n, seed, q)
    return out


def u64_and(n: int, seed: int, q: int, out: np.ndarray | None = None) -> np.ndarray:
    out = np.empty(n, np.uint64) if out is None else out
    _load().wl_u64_and(_ptr(out), n, seed, q)
    return out


def u32_const(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, np.uint32)
    _load().wl_u32_const(_ptr(out), n, seed)
    return out


def u64_const(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, np.uint64)
    _load().wl_u64_const(_ptr(out), n, seed)
    return out


def f32_normal_bits(n: int, seed: int) -> np.ndarray:
    """Raw IEEE-754 bits (uint32) of the float32 N(0,1) workload."""
    out = np.empty(n, np.uint32)
    _load().wl_f32_normal(_ptr(out), n, seed)
    return out


def f64_normal_bits(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, np.uint64)
    _load().wl_f64_normal(_ptr(out), n, seed)
    return out


def iota_u32(n: int) -> np.ndarray:
    out = np.empty(n, np.uint32)
    _load().wl_iota_u32(_ptr(out), n)
    return out


def uniform01(n: int, seed: int, stream: int = 0) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().wl_uniform01(_ptr(out), n, seed, stream)
    return out


def normal(n: int, seed: int, stream: int = 0) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().wl_normal(_ptr(out), n, seed, stream)
    return out


KEY_TYPES = ("u32", "u64", "f32", "f64", "i32", "i64")
DISTRIBUTIONS = ("uniform", "and2", "and3", "and4", "and5", "and8", "and16", "const", "normal")


def keys(key_type: str, dist: str, n: int, seed: int) -> np.ndarray:
    """Key bits for ``key_type`` (uint32 for 32-bit types, uint64 for 64-bit)."""
    wide = key_type in ("u64", "f64", "i64")
    if dist == "normal":
        if key_type == "f32":
            return f32_normal_bits(n, seed)
        if key_type == "f64":
            return f64_normal_bits(n, seed)
        raise ValueError("normal keys are float keys")
    if dist == "const":
        return u64_const(n, seed) if wide else u32_const(n, seed)
    if dist == "uniform":
        q = 1
    elif dist.startswith("and"):
        q = int(dist[3:])
    else:
        raise ValueError(f"unknown distribution {dist!r}")
    return u64_and(n, seed, q) if wide else u32_and(n, seed, q)


def segment_sizes(num_segments: int, seed: int, median: float = 32768.0, sigma: float = 1.18,
                  lo: int = 1024, hi: int = 4 << 20) -> np.ndarray:
    """Lognormal segment lengths (median ``median``, log-sd ``sigma``) clipped to [lo, hi]."""
    z = normal(num_segments, seed, stream=7)
    sizes = np.rint(median * np.exp(sigma * z))
    return np.clip(sizes, lo, hi).astype(np.int64)


def entropy_per_bit(q: int) -> float:
    """Shannon entropy per key bit when each bit is set with probability 2^-q (Table 1)."""
    p = 2.0 ** (-q)
    if p >= 1.0 or p <= 0.0:
        return 0.0
    return float(-(p * np.log2(p) + (1 - p) * np.log2(1 - p)))
