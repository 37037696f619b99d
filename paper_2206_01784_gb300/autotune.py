"""Autotuner for the binning kernel's variants and digit width.

The library carries os_num_tile_configs() variants of the digit-binning kernel
(tile geometry - threads per block and keys per thread - times the digit
ranking method) and digit widths d of 5 to 8 bits (Section 4, Table 2: fewer
bits make each pass cheaper and the sort longer), and keeps one active
(variant, d) per (key width, payload, size bucket). ``tune`` times every
variant at d = 8 and variant 4 (the one narrower digits run) at each smaller
d on seeded uniform keys of a size representative of each bucket (CUDA events
around whole sorts), installs the fastest through os_set_tile_config_bucket
and os_set_radix_bits_bucket and returns the table; ``save`` / ``load`` /
``apply`` keep tables across processes. Results of a sort never depend on the
variant or on d - only its speed does - and workspaces are sized for the
smallest tile and the most places, so a table can be applied at any time
between calls.
"""
from __future__ import annotations

import json
import os

from . import onesweep as osw
from . import workload

# representative sort size of each size bucket (n < 2^16, < 2^20, < 2^24, larger)
BUCKET_SIZES = {0: 1 << 15, 1: 1 << 19, 2: 1 << 23, 3: 1 << 26}


NARROW_VARIANT = 4          # the tile variant of digits narrower than 8 bits
RADIX_BITS = (5, 6, 7, 8)  # digit widths the library carries


def _time_sort(kt, k, v, ko, vo, n, kb, ws, steps, warmup, torch, cfg=None, radix_bits=None):
    s = torch.cuda.current_stream()
    sp = s.cuda_stream

    def one():
        if v is None:
            rc = osw.os_sort_keys_ex(kt, k.data_ptr(), ko.data_ptr(), n, 0, kb, ws.data_ptr(), ws.numel(), sp,
                                     tile_config=cfg, radix_bits=radix_bits)
        else:
            rc = osw.os_sort_pairs_ex(kt, k.data_ptr(), ko.data_ptr(), v.data_ptr(), vo.data_ptr(), n, 0, kb,
                                      ws.data_ptr(), ws.numel(), sp, tile_config=cfg, radix_bits=radix_bits)
        if rc != osw.OS_OK:
            raise osw.OnesweepError(rc, "autotune sort")

    for _ in range(warmup):
        one()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        one()
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def candidates(radix_bits=RADIX_BITS):
    """(tile variant, digit width) pairs the tuner times: every variant with
    8-bit digits, and the narrow-digit variant at each smaller width."""
    out = [(cfg, 8) for cfg in range(osw.os_num_tile_configs())] if 8 in radix_bits else []
    return out + [(NARROW_VARIANT, d) for d in sorted(radix_bits) if d != 8]


def tune(key_bits=(32, 64), value_bytes=(0, 4), buckets=None, steps: int = 5, warmup: int = 2, seed: int = 1234,
         sizes: dict | None = None, verbose: bool = False, radix_bits=RADIX_BITS) -> dict:
    """Times every candidate and installs the fastest per (key bits, value bytes, bucket).

    Returns {(key_bits, value_bytes, bucket): {"cfg": variant, "radix_bits": d,
    "ms": {"cfg/d": ms}, "n": keys}}."""
    import numpy as np
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    sizes = dict(BUCKET_SIZES, **(sizes or {}))
    buckets = list(range(osw.os_num_size_buckets())) if buckets is None else list(buckets)
    table = {}
    for kb in key_bits:
        kt = osw.OS_KEY_U32 if kb == 32 else osw.OS_KEY_U64
        for vb in value_bytes:
            for b in buckets:
                n = sizes[b]
                keys = workload.keys("u32" if kb == 32 else "u64", "uniform", n, seed + b)
                k = torch.from_numpy(keys.view(np.int32 if kb == 32 else np.int64)).to(dev)
                ko = torch.empty_like(k)
                v = vo = None
                if vb:
                    v = torch.from_numpy(workload.iota_u32(n).view(np.int32)).to(dev)
                    vo = torch.empty_like(v)
                ws = osw.workspace(kt, n, vb, 0, kb, dev)
                times = {}
                for cfg, d in candidates(radix_bits):
                    times[(cfg, d)] = _time_sort(kt, k, v, ko, vo, n, kb, ws, steps, warmup, torch, cfg, d)
                best = min(times, key=times.__getitem__)
                osw.os_set_tile_config_bucket(kb, vb, b, best[0])
                osw.os_set_radix_bits_bucket(kb, vb, b, best[1])
                table[(kb, vb, b)] = {"cfg": best[0], "radix_bits": best[1],
                                      "ms": {f"{c}/{d}": t for (c, d), t in times.items()}, "n": n}
                if verbose:
                    print(f"key_bits={kb} value_bytes={vb} bucket={b} n={n}: variant {best[0]}, {best[1]}-bit "
                          f"digits ({times[best]:.3f} ms)", flush=True)
                del k, ko, v, vo, ws
    return table


def apply(table: dict) -> None:
    """Installs a table from ``tune`` or ``load``."""
    for (kb, vb, b), rec in table.items():
        rc = osw.os_set_tile_config_bucket(kb, vb, b, int(rec["cfg"]))
        if rc != osw.OS_OK:
            raise osw.OnesweepError(rc, "os_set_tile_config_bucket")
        rc = osw.os_set_radix_bits_bucket(kb, vb, b, int(rec.get("radix_bits", 8)))
        if rc != osw.OS_OK:
            raise osw.OnesweepError(rc, "os_set_radix_bits_bucket")


def current() -> dict:
    """The active variant of every (key bits, value bytes, bucket)."""
    return {(kb, vb, b): {"cfg": osw.os_get_tile_config_bucket(kb, vb, b),
                          "radix_bits": osw.os_get_radix_bits_bucket(kb, vb, b)}
            for kb in (32, 64) for vb in (0, 4) for b in range(osw.os_num_size_buckets())}


def save(table: dict, path: str, device_name: str = "") -> None:
    rows = [{"key_bits": kb, "value_bytes": vb, "bucket": b, **rec} for (kb, vb, b), rec in sorted(table.items())]
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "w") as f:
        json.dump({"device": device_name, "variants": osw.os_num_tile_configs(), "table": rows}, f, indent=1)


def load(path: str) -> dict:
    with open(path) as f:
        data = json.load(f)
    if data.get("variants") != osw.os_num_tile_configs():
        raise ValueError("table was tuned for a different set of kernel variants")
    return {(r["key_bits"], r["value_bytes"], r["bucket"]): {k: v for k, v in r.items()
                                                               if k not in ("key_bits", "value_bytes", "bucket")}
            for r in data["table"]}
