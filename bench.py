#!/usr/bin/env python
"""Throughput of the GB300 Onesweep sort (arXiv 2206.01784) on 256M uint32
keys with uint32 index values, the paper's Section 4 workload shape (seeded,
synthetic, uniform random keys).

One step = one full sort through the C ABI (os_sort_pairs): the header memset,
the all-places histogram + exclusive sum, and 4 chained-scan binning passes.
Inputs (2 GiB of keys + values) are resident in HBM and far larger than L2, so
no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torchrun) every rank sorts its own array of the same
size: independent replicas, weak scaling, no collective on the data path.
``--impl reference`` times the CPU oracle instead (rank 0 only).
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GKeys/s @256M u32 keys, % HBM roofline; batched vs per-array GKeys/s, p99 ms"
UNIT = "GKeys/s"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--log2n", type=int, default=None,
                   help="keys per GPU = 2^log2n (default 28; 27 for 64-bit keys, the u64 configuration)")
    p.add_argument("--key-type", choices=["u32", "u64", "f32", "f64", "i32", "i64"], default="u32")
    p.add_argument("--dist", default="uniform")
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--serve-sweep", default="0.5,0.9",
                   help="other offered loads (fractions of the measured capacity) for the serving stream")
    p.add_argument("--e2e-lanes", type=int, default=3, help="streams (each with a device workspace) the end-to-end calls rotate over")
    p.add_argument("--keys-only", action="store_true", help="sort keys without values")
    p.add_argument("--host-copy-mode", choices=["default", "engines", "link"], default="default",
                   help="how the end-to-end host-buffer calls move data (os_set_host_copy_mode)")
    p.add_argument("--no-extras", action="store_true", help="skip the batched and serving measurements")
    p.add_argument("--serve-requests", type=int, default=10000)
    p.add_argument("--no-std-full", action="store_true",
                   help="time std::stable_sort on 2^24 pairs only (not on the whole workload)")
    p.add_argument("--tile-config", type=int, default=None,
                   help="binning variant for the timed sorts (os_set_tile_config; default: the library's choice)")
    args = p.parse_args()
    if args.log2n is None:
        args.log2n = 27 if args.key_type in ("u64", "f64", "i64") else 28
    if args.key_type in ("f32", "f64") and args.dist == "uniform":
        args.dist = "normal"  # the float workload: N(0,1) with signed zeros and duplicates
    return args


KEY_BITS = {"u32": 32, "u64": 64, "f32": 32, "f64": 64, "i32": 32, "i64": 64}


def order_key(torch, t, key_type):
    """int64 tensor whose signed order is the sort order of key_type's bits
    (t: int32 or int64 tensor holding the bits), for the sanity check."""
    if key_type in ("u32", "i32", "f32"):
        x = t.to(torch.int32)
        if key_type == "f32":  # sign-flip: negative floats all bits inverted, others sign bit set
            x = x ^ ((x >> 31) | torch.tensor(-(1 << 31), dtype=torch.int32, device=t.device))
        x64 = x.to(torch.int64)
        return x64 if key_type == "i32" else x64 & 0xFFFFFFFF
    x = t.to(torch.int64)
    smin = torch.tensor(-(1 << 63), dtype=torch.int64, device=t.device)
    if key_type == "f64":
        x = x ^ ((x >> 63) | smin)
    return x if key_type == "i64" else x ^ smin


def workload_name(n, dist, seed, pairs=True, key_type="u32"):
    size = f"{n >> 20}M" if n >= (1 << 20) else str(n)
    payload = " + u32 index values" if pairs else " only"
    return f"{size} {key_type} keys{payload}, {dist} keys (seed {seed})"


# The sources the timed binning kernel is compiled from: a profile's traffic
# figure stays valid while these are unchanged.
KERNEL_SOURCES = ("os_common.cuh", "os_internal.h", "os_binning.cuh", "os_bin32_pairs_f0_single.cu")


def source_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2206_01784_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_tag: str, n: int):
    """DRAM bytes per launch from a committed ncu summary whose source hash
    matches the current kernels (None when absent or stale)."""
    want = source_hash()
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")) + glob.glob(os.path.join(ROOT, "profiles", "*.txt"))):
        fields = {}
        for line in open(f):
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
        if fields.get("kernel_tag") == kernel_tag and fields.get("source_hash") == want:
            try:
                per_key = float(fields["dram_bytes_per_key"])
            except (KeyError, ValueError):
                continue
            return per_key * n
    return None


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", self.gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_smi_id(torch, dev_index: int) -> str:
    try:
        uuid = str(torch.cuda.get_device_properties(dev_index).uuid)
        if uuid:
            return uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        return vis.split(",")[dev_index]
    return str(dev_index)


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def time_oracle(n: int, dist: str, seed: int, repeats: int = 1, key_type: str = "u32"):
    """The CPU oracle as it stands (single thread), on n pairs of the workload."""
    import oracle
    from paper_2206_01784_gb300 import workload

    keys = workload.keys(key_type, dist, n, seed)
    vals = workload.iota_u32(n)
    times = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        oracle.sort(key_type, keys, vals)
        times.append(time.perf_counter() - t0)
    return times


def time_cpu_baselines(keys_np, vals_np, key_type: str, full_std: bool = True):
    """The CPU comparison rows on this host (not the oracle; checked against it
    by tests/test_cpu_baselines.py): the multi-threaded LSD radix sort on all
    host threads over the whole workload, and std::stable_sort on one thread
    over its first 2^24 pairs and (full_std) the whole workload."""
    import oracle

    n = keys_np.size
    threads = oracle.hardware_threads()
    t0 = time.perf_counter()
    oracle.parallel_sort(key_type, keys_np, vals_np, threads=threads)
    t_par = time.perf_counter() - t0
    rows = {"parallel_lsd": {"value": n / t_par / 1e9, "unit": UNIT, "threads": threads, "seconds": t_par,
                             "sample": f"the whole workload ({n} pairs), 8-bit places, all host threads"}}
    std = {}
    sizes = [min(n, 1 << 24)] + ([n] if full_std and n > (1 << 24) else [])
    for m in sizes:
        t0 = time.perf_counter()
        oracle.std_stable_sort(key_type, keys_np[:m], vals_np[:m])
        dt = time.perf_counter() - t0
        std[f"n={m}"] = {"value": m / dt / 1e9, "unit": UNIT, "seconds": dt, "threads": 1}
    rows["std_stable_sort"] = std
    return rows


def measure_config(torch, osw, workload, np, dev, key_type: str, log2n: int, pairs: bool, dist: str, seed: int,
                   steps: int = 10, warmup: int = 3, radix_bits: int = 8):
    """One more workload configuration through os_sort_pairs_ex /
    os_sort_keys_ex, timed like the headline (CUDA events around the steps,
    launch times from the library's profile hooks): GKeys/s, ms per step, the
    binning kernel's and the whole step's fraction of the HBM roofline.
    radix_bits: bits per digit place."""
    n = 1 << log2n
    bits = KEY_BITS[key_type]
    kbytes = bits // 8
    kview = np.int64 if bits == 64 else np.int32
    keys = torch.from_numpy(workload.keys(key_type, dist, n, seed).view(kview)).to(dev)
    vals = torch.from_numpy(workload.iota_u32(n).view(np.int32)).to(dev) if pairs else None
    ko = torch.empty_like(keys)
    vo = torch.empty_like(vals) if pairs else None
    kt = osw.KEY_TYPES[key_type]
    lay = osw.os_sort_workspace_layout(kt, n, 4 if pairs else 0, 0, bits)
    ws = torch.empty(lay.total_bytes, dtype=torch.uint8, device=dev)
    sp = torch.cuda.current_stream(dev).cuda_stream

    places = (bits + radix_bits - 1) // radix_bits

    def step():
        if pairs:
            rc = osw.os_sort_pairs_ex(kt, keys.data_ptr(), ko.data_ptr(), vals.data_ptr(), vo.data_ptr(), n, 0, bits,
                                      ws.data_ptr(), ws.numel(), sp, radix_bits=radix_bits)
        else:
            rc = osw.os_sort_keys_ex(kt, keys.data_ptr(), ko.data_ptr(), n, 0, bits, ws.data_ptr(), ws.numel(), sp,
                                     radix_bits=radix_bits)
        if rc != osw.OS_OK:
            raise osw.OnesweepError(rc, "sort")

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    cap = steps * (places + 1) + 16
    osw.os_profile_start(cap)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    _, _, recs = osw.os_profile_stop(cap)
    if osw.os_workspace_status(ws.data_ptr(), sp) != osw.OS_OK:
        raise RuntimeError("device status after the configuration's steps")
    ok64 = order_key(torch, ko, key_type)
    if not bool((ok64[1:] >= ok64[:-1]).all().item()):
        raise RuntimeError("configuration output not sorted")
    peak, _ = hbm_peak()
    bin_ms = statistics.mean([m for k, _, m in recs if k == 1])
    hist_ms = statistics.mean([m for k, _, m in recs if k == 0])
    per_pass = n * 2 * (kbytes + (4 if pairs else 0))
    step_bytes = n * kbytes + places * per_pass
    return {"workload": workload_name(n, dist, seed, pairs, key_type), "keys": n, "places": places,
            "radix_bits": radix_bits, "gkeys_per_s": n / ms / 1e6, "ms_per_step": ms, "binning_avg_ms": bin_ms,
            "histogram_avg_ms": hist_ms, "binning_frac": per_pass / (bin_ms / 1e3) / 1e9 / peak,
            "step_frac": step_bytes / (ms / 1e3) / 1e9 / peak, "steps": steps}


# Section 4, Table 2 (A100, 256M random u32 keys only): digit width d ->
# (histogram us, partition us per pass); context for the GB300 sweep.
PAPER_TABLE2_A100 = {5: (652, 1573), 6: (653, 1685), 7: (679, 1812), 8: (747, 1995), 9: (655, 2541)}


def measure_digit_widths(torch, osw, workload, np, dev, log2n: int = 28, steps: int = 5):
    """Table 2's sweep on this GPU: 2^log2n uniform u32 keys only, sorted with
    d = 5..8 bits per digit place; per d the histogram and per-pass binning
    times (us), the per-bit cost of a pass and the whole sort."""
    rows = {}
    for d in (5, 6, 7, 8):
        r = measure_config(torch, osw, workload, np, dev, "u32", log2n, False, "uniform", 1, steps=steps, radix_bits=d)
        rows[str(d)] = {"passes": r["places"], "histogram_us": r["histogram_avg_ms"] * 1e3,
                        "partition_us": r["binning_avg_ms"] * 1e3, "partition_per_bit_us": r["binning_avg_ms"] * 1e3 / d,
                        "sort_ms": r["ms_per_step"], "gkeys_per_s": r["gkeys_per_s"], "binning_frac": r["binning_frac"]}
        torch.cuda.empty_cache()
    return {"workload": workload_name(1 << log2n, "uniform", 1, False, "u32"), "rows": rows,
            "paper_a100_us": {str(d): {"histogram_us": h, "partition_us": p, "partition_per_bit_us": round(p / d)}
                              for d, (h, p) in PAPER_TABLE2_A100.items()}}


def measure_copy_ceiling(torch, dev, nbytes: int):
    """Plain cudaMemcpyAsync rates between pinned host memory and the device
    on this machine: host-to-device, device-to-host, and both at once on two
    streams (GB/s) - the ceiling for an end-to-end sort that moves its inputs
    up and its result down."""
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h2 = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d2 = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize(dev)
        return (time.perf_counter() - t0) / reps

    def up():
        with torch.cuda.stream(s1):
            d.copy_(h, non_blocking=True)

    def down():
        with torch.cuda.stream(s1):
            h.copy_(d, non_blocking=True)

    def both():
        with torch.cuda.stream(s1):
            d.copy_(h, non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(d2, non_blocking=True)

    t_up, t_down, t_both = timed(up), timed(down), timed(both)
    return {"h2d_gbs": nbytes / t_up / 1e9, "d2h_gbs": nbytes / t_down / 1e9,
            "both_directions_gbs_each": nbytes / t_both / 1e9, "bytes_per_copy": nbytes,
            "api": "cudaMemcpyAsync (torch copy_) from/to pinned host memory"}


def run_reference(args):
    """Reference arm: the CPU oracle timed on the host cores, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    # bounded sample per step (a slice of the 2^28 workload): about a minute
    # of CPU work in total at the oracle's ~14 Mkeys/s, at most 2^22 per step
    n = 1 << 22
    while n > (1 << 16) and n * (args.steps + args.warmup) > 840_000_000:
        n >>= 1
    times = time_oracle(n, args.dist, args.seed, repeats=args.warmup + args.steps, key_type=args.key_type)[args.warmup:]
    total = sum(times)
    value = n * len(times) / total / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / len(times) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.key_type, "data": "synthetic", "impl": "reference",
        "config": {"workload": workload_name(1 << args.log2n, args.dist, args.seed, key_type=args.key_type),
                   "sample_keys_per_step": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{n} {args.key_type} pairs of the same distribution per step, single-threaded C oracle",
                         "cpu": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_batch(torch, osw, workload, np, dev, steps: int = 20):
    """4096 lognormal segments (median 32K keys, clipped 1K-4M, seed 10) of u32
    keys + u32 values: one graph-captured os_sort_batch against one
    os_sort_pairs call per segment on one stream; outputs must be identical."""
    sizes = workload.segment_sizes(4096, seed=10)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offs[-1])
    keys = workload.keys("u32", "uniform", n, 10)
    k = torch.from_numpy(keys.view(np.int32)).to(dev)
    v = torch.from_numpy(workload.iota_u32(n).view(np.int32)).to(dev)
    o = torch.from_numpy(offs).to(dev)
    bk, bv = torch.empty_like(k), torch.empty_like(v)
    ws = osw.batch_workspace(osw.OS_KEY_U32, n, len(sizes), 4, 0, 32, dev)
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        osw.sort_batch(k, o, v, key_type="u32", keys_out=bk, values_out=bv, ws=ws)  # warm-up before capture
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        osw.sort_batch(k, o, v, key_type="u32", keys_out=bk, values_out=bv, ws=ws)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        g.replay()
    e1.record()
    torch.cuda.synchronize(dev)
    t_batch = e0.elapsed_time(e1) / steps
    pk, pv = torch.empty_like(k), torch.empty_like(v)
    wss = osw.workspace(osw.OS_KEY_U32, int(sizes.max()), 4, 0, 32, dev)
    sp = torch.cuda.current_stream(dev).cuda_stream

    def per_array():
        for i in range(len(sizes)):
            lo, hi = int(offs[i]), int(offs[i + 1])
            rc = osw.os_sort_pairs(osw.OS_KEY_U32, k.data_ptr() + 4 * lo, pk.data_ptr() + 4 * lo,
                                   v.data_ptr() + 4 * lo, pv.data_ptr() + 4 * lo, hi - lo, 0, 32, wss.data_ptr(),
                                   wss.numel(), sp)
            if rc != osw.OS_OK:
                raise osw.OnesweepError(rc, "os_sort_pairs")

    per_array()
    torch.cuda.synchronize(dev)
    e0.record()
    per_array()
    per_array()
    e1.record()
    torch.cuda.synchronize(dev)
    t_per = e0.elapsed_time(e1) / 2
    identical = bool(torch.equal(bk, pk) and torch.equal(bv, pv))
    if not identical:
        raise RuntimeError("batched output differs from per-array output")
    return {"workload": "4096 segments, lognormal sizes (median 32K, sigma 1.18, clipped 1K-4M), u32 keys + u32 "
                        "values, uniform keys (seed 10)", "keys": n, "segments": len(sizes),
            "batched_gkeys_per_s": n / t_batch / 1e6, "batched_ms": t_batch, "cuda_graph": True,
            "per_array_gkeys_per_s": n / t_per / 1e6, "per_array_ms": t_per, "speedup": t_per / t_batch,
            "identical_output": identical, "tile_variant": osw.os_get_tile_config_bucket(32, 4, osw.os_size_bucket(n // len(sizes)))}


def measure_serving(torch, dev, count: int, sweep_loads=()):
    """Continuous batching of a Poisson request stream (sizes log-uniform
    16K-64M keys, key types 60/25/15 % u32/u64/f32 with u32 values, 40 GB
    device budget, seed 11), two ways: request data copied from pinned host
    memory per request (the service the host link bounds), and request data
    already in device memory (the service the sorts bound). For each: the
    capacity (every request present at once), then the stream offered in real
    time at 0.7x that capacity and at the sweep's other loads; p50/p99 latency
    from arrival to completion and requests per batch at every load."""
    from paper_2206_01784_gb300 import serve

    def one(resident: bool):
        srv = serve.Server(budget_bytes=40 * 10**9, device=dev, device_resident=resident)
        probe = serve.make_requests(count, seed=11, rate_per_s=1.0)
        for r in probe:
            r.arrival = 0.0
        cap = srv.run(probe, realtime=False)
        mean_keys = sum(r.n for r in probe) / len(probe)
        capacity_rps = cap["gkeys_per_s"] * 1e9 / mean_keys
        out = {"capacity_gkeys_per_s": cap["gkeys_per_s"], "capacity_mean_batch_requests": cap["mean_batch_requests"]}
        loads = []
        for load in (0.7,) + tuple(sweep_loads):
            st = srv.run(serve.make_requests(count, seed=11, rate_per_s=load * capacity_rps), realtime=True)
            loads.append({"load": load, "offered_requests_per_s": load * capacity_rps, "gkeys_per_s": st["gkeys_per_s"],
                          "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                          "tail_wait_ms": st["tail_wait_ms"], "tail_service_ms": st["tail_service_ms"],
                          "batches": st["batches"], "mean_batch_requests": st["mean_batch_requests"]})
        out["loads"] = loads
        del srv
        torch.cuda.empty_cache()
        return out

    host = one(False)
    resident = one(True)
    at07 = host["loads"][0]
    return {"workload": f"{count} requests, Poisson arrivals, sizes log-uniform 16K-64M, u32/u64/f32 keys 60/25/15 % "
                        "+ u32 values, 40 GB budget, seed 11; offered at 0.7x (and the sweep's loads) of each "
                        "service's measured capacity",
            # the headline service (inputs copied from pinned host memory), as before
            "capacity_gkeys_per_s": host["capacity_gkeys_per_s"], "gkeys_per_s": at07["gkeys_per_s"],
            "p50_ms": at07["p50_ms"], "p99_ms": at07["p99_ms"], "mean_batch_requests": at07["mean_batch_requests"],
            "host_inputs": host, "device_resident": resident}


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2206_01784_gb300 import onesweep as osw
    from paper_2206_01784_gb300 import workload

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    osw.load()
    if args.host_copy_mode != "default":
        osw.os_set_host_copy_mode(osw.OS_HOST_COPY_LINK if args.host_copy_mode == "link" else osw.OS_HOST_COPY_ENGINES)
    n = 1 << args.log2n
    if args.tile_config is not None:
        for vb in (0, 4):
            rc = osw.os_set_tile_config(KEY_BITS[args.key_type], vb, args.tile_config)
            if rc != osw.OS_OK:
                raise osw.OnesweepError(rc, "os_set_tile_config")
    seed = args.seed + 1000 * rank
    bits = KEY_BITS[args.key_type]
    kbytes = bits // 8
    kview = np.int64 if bits == 64 else np.int32
    keys_np = workload.keys(args.key_type, args.dist, n, seed)
    vals_np = workload.iota_u32(n)
    keys = torch.from_numpy(keys_np.view(kview)).to(dev)
    vals = torch.from_numpy(vals_np.view(np.int32)).to(dev)
    keys_out = torch.empty_like(keys)
    vals_out = torch.empty_like(vals)
    kt = osw.KEY_TYPES[args.key_type]
    pairs = not args.keys_only
    lay = osw.os_sort_workspace_layout(kt, n, 4 if pairs else 0, 0, bits)
    ws = torch.empty(lay.total_bytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    def step():
        if pairs:
            rc = osw.os_sort_pairs(kt, keys.data_ptr(), keys_out.data_ptr(), vals.data_ptr(), vals_out.data_ptr(), n,
                                   0, bits, ws.data_ptr(), ws.numel(), sp)
        else:
            rc = osw.os_sort_keys(kt, keys.data_ptr(), keys_out.data_ptr(), n, 0, bits, ws.data_ptr(), ws.numel(), sp)
        if rc != osw.OS_OK:
            raise osw.OnesweepError(rc, "os_sort_pairs" if pairs else "os_sort_keys")

    warmup = max(args.warmup, 3)
    for _ in range(warmup):
        step()
    barrier()

    sampler = ClockSampler(gpu_smi_id(torch, local))
    sampler.start()
    time.sleep(0.3)
    strips = -(-n // ((1 << 30) - 1))  # passes over 2^30 keys or more run in strips
    capacity = args.steps * (lay.num_places * strips + 1) + 16
    osw.os_profile_start(capacity)
    barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        step()
    t_end.record(stream)
    barrier()
    elapsed_ms = t_start.elapsed_time(t_end)
    prof_rc, launches, recs = osw.os_profile_stop(capacity)
    clocks = sampler.stop()
    status = osw.os_workspace_status(ws.data_ptr(), sp)
    if status != osw.OS_OK:
        raise osw.OnesweepError(status, "device status after timed steps")

    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    ms_per_step = max_ms / args.steps
    value = world * n * args.steps / (max_ms / 1e3) / 1e9

    # sanity: output sorted and values a permutation carrying their keys (outside the timed region)
    ko64 = order_key(torch, keys_out, args.key_type)
    ok = bool((ko64[1:] >= ko64[:-1]).all().item())
    del ko64
    if pairs:
        gathered = keys[vals_out.to(torch.int64)]
        ok = ok and bool(torch.equal(gathered, keys_out))
        del gathered
    if not ok:
        raise RuntimeError("sorted output failed the sanity check")

    # roofline of the dominant kernel (the binning pass)
    peak, peak_kind = hbm_peak()
    bin_ms = [ms for k, _, ms in recs if k == 1]
    hist_ms = [ms for k, _, ms in recs if k == 0]
    bin_avg = statistics.mean(bin_ms)
    bytes_per_pass = n * 2 * (kbytes + (4 if pairs else 0))
    achieved = bytes_per_pass / (bin_avg / 1e3) / 1e9
    traffic = profiled_traffic(f"binning_{args.key_type}_{'pairs' if pairs else 'keys'}", n)
    step_bytes = n * kbytes + lay.num_places * bytes_per_pass
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": f"binning_kernel<{bits}, {'pairs' if pairs else 'keys'}>",
                "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": bytes_per_pass, "avg_launch_ms": bin_avg}
    step_roofline = {"achieved": step_bytes / (ms_per_step / 1e3) / 1e9, "peak": peak,
                     "frac": step_bytes / (ms_per_step / 1e3) / 1e9 / peak, "algorithmic_bytes_per_step": step_bytes,
                     "histogram_avg_ms": statistics.mean(hist_ms) if hist_ms else None,
                     "binning_avg_ms": bin_avg}

    # End to end through the C ABI's host-buffer entry point: every step's
    # call uploads its keys (and values) from pinned host memory, sorts them
    # and downloads the sorted result into pinned host memory. Calls rotate
    # over three streams with a device workspace each, so one array's upload,
    # another's sort and a third's download overlap, the way a stream of
    # arrays would be served.
    e2e = None
    if args.e2e_steps > 0:
        hk = torch.from_numpy(keys_np.view(kview)).pin_memory()
        hv = torch.from_numpy(vals_np.view(np.int32)).pin_memory()
        lanes = max(1, args.e2e_lanes)
        hko = [torch.empty_like(hk).pin_memory() for _ in range(lanes)]
        hvo = [torch.empty_like(hv).pin_memory() for _ in range(lanes)]
        hws = osw.os_sort_host_workspace_bytes(kt, n, 4 if pairs else 0, 0, bits)
        wss = [torch.empty(hws, dtype=torch.uint8, device=dev) for _ in range(lanes)]
        streams = [torch.cuda.Stream(dev) for _ in range(lanes)]

        def e2e_step(i):
            b = i % lanes
            sp_b = streams[b].cuda_stream
            if pairs:
                rc = osw.os_sort_pairs_host(kt, hk.data_ptr(), hko[b].data_ptr(), hv.data_ptr(), hvo[b].data_ptr(),
                                            n, 0, bits, wss[b].data_ptr(), hws, sp_b)
            else:
                rc = osw.os_sort_keys_host(kt, hk.data_ptr(), hko[b].data_ptr(), n, 0, bits, wss[b].data_ptr(), hws,
                                           sp_b)
            if rc != osw.OS_OK:
                raise osw.OnesweepError(rc, "sort (host buffers)")

        def timed_e2e():
            for i in range(lanes):
                e2e_step(i)
            torch.cuda.synchronize(dev)
            barrier()
            e0 = [torch.cuda.Event(enable_timing=True) for _ in range(lanes)]
            e1 = [torch.cuda.Event(enable_timing=True) for _ in range(lanes)]
            t0 = time.perf_counter()
            for b in range(lanes):
                e0[b].record(streams[b])
            for i in range(args.e2e_steps):
                e2e_step(i)
            for b in range(lanes):
                e1[b].record(streams[b])
            torch.cuda.synchronize(dev)
            barrier()
            wall_ms = (time.perf_counter() - t0) * 1e3
            et_ms = max(max(e0[a].elapsed_time(e1[b]) for a in range(lanes) for b in range(lanes)), 0.0)
            et = torch.tensor([max(et_ms, wall_ms)], dtype=torch.float64, device=dev)
            if world > 1:
                dist.all_reduce(et, op=dist.ReduceOp.MAX)
            for b in range(lanes):
                st = osw.os_workspace_status(wss[b].data_ptr(), streams[b].cuda_stream)
                if st != osw.OS_OK:
                    raise osw.OnesweepError(st, "device status after the end-to-end steps")
            last = (args.e2e_steps - 1) % lanes
            ok = np.array_equal(hko[last].numpy()[:: 1 << 16], keys_out.cpu().numpy()[:: 1 << 16])
            if not ok:
                raise RuntimeError("end-to-end result differs from the device result")
            return world * n * args.e2e_steps / (float(et.item()) / 1e3) / 1e9

        # the library's default copy mode gives the headline figure; the other
        # mode (copy kernels over the host link, or the copy engines) is timed
        # beside it on one GPU
        mode_names = {osw.OS_HOST_COPY_ENGINES: "copy engines (cudaMemcpyAsync)",
                      osw.OS_HOST_COPY_LINK: "copy kernels reading and writing the mapped host buffers"}
        default_mode = osw.os_get_host_copy_mode()
        e2e = {"value": timed_e2e(), "unit": UNIT,
               "h2d_bytes_per_step": hk.numel() * kbytes + (hv.numel() * 4 if pairs else 0),
               "d2h_bytes_per_step": hk.numel() * kbytes + (hv.numel() * 4 if pairs else 0), "steps": args.e2e_steps,
               "api": "os_sort_pairs_host" if pairs else "os_sort_keys_host",
               "pipelined": f"calls rotate over {lanes} streams with a device workspace each",
               "copies": mode_names[default_mode]}
        if world == 1 and not args.no_extras:
            other = osw.OS_HOST_COPY_LINK if default_mode == osw.OS_HOST_COPY_ENGINES else osw.OS_HOST_COPY_ENGINES
            osw.os_set_host_copy_mode(other)
            try:
                e2e["other_copy_mode"] = {"copies": mode_names[other], "value": timed_e2e()}
            finally:
                osw.os_set_host_copy_mode(default_mode)

    batched = serving = configs = copy_ceiling = digit_widths = None
    if world == 1 and not args.no_extras:
        # the other workload configurations at full size (extras, not the headline)
        configs = {}
        for name, kt_, log2n_, pairs_, dist_, seed_ in (("keys_only_256m_u32", "u32", 28, False, "uniform", 1),
                                                        ("u64_pairs_128m", "u64", 27, True, "uniform", 8),
                                                        ("f32_pairs_256m", "f32", 28, True, "normal", 9)):
            configs[name] = measure_config(torch, osw, workload, np, dev, kt_, log2n_, pairs_, dist_, seed_)
            torch.cuda.empty_cache()
        digit_widths = measure_digit_widths(torch, osw, workload, np, dev)
        copy_ceiling = measure_copy_ceiling(torch, dev, n * (kbytes + (4 if pairs else 0)))
        if e2e is not None:
            moved = e2e["h2d_bytes_per_step"] + e2e["d2h_bytes_per_step"]
            copy_ceiling["e2e_bound_gkeys_per_s"] = n / (moved / 2 / (copy_ceiling["both_directions_gbs_each"] * 1e9)) / 1e9
        batched = measure_batch(torch, osw, workload, np, dev)
        if args.serve_requests > 0:
            loads = [float(x) for x in args.serve_sweep.split(",") if x.strip()]
            serving = measure_serving(torch, dev, args.serve_requests, loads)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = n // 2
        times = time_oracle(sample, args.dist, seed, key_type=args.key_type)
        cpu = {"value": sample / times[0] / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{sample} {args.key_type} pairs (half the workload, same distribution), single-threaded C oracle, "
                         f"{times[0]:.1f} s", "cpu": cpu_model(), "nproc": os.cpu_count()}
        # comparison rows on the same host cores (not the oracle)
        cpu.update(time_cpu_baselines(keys_np, vals_np, args.key_type, full_std=not args.no_std_full))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.key_type, "data": "synthetic",
            "config": {"workload": workload_name(n, args.dist, args.seed, pairs, args.key_type), "keys_per_gpu": n,
                       "key_type": args.key_type, "values": "u32 (input index)" if pairs else None, "bits": [0, bits],
                       "places": lay.num_places, "tile_keys": lay.tile_keys, "parallelism": f"replicas x{world}",
                       "l2": f"no flush: {n * (kbytes + (4 if pairs else 0)) / 2**30:.2f} GiB of inputs per step, "
                             "larger than L2"},
            "roofline": roofline, "roofline_step": step_roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks, "gpu": torch.cuda.get_device_name(dev),
            "batched": batched, "serving": serving, "configs": configs, "digit_widths": digit_widths,
            "copy_ceiling": copy_ceiling,
            "paper_context": "A100-80GB: 29.4 GKey/s, 256M u32 keys only (different hardware and workload)",
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
