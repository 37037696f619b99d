"""bench.py's host-side parts, without a GPU: the reference arm (the CPU
oracle timed on a bounded sample) prints one JSON line with the contract's
keys; non-zero ranks print nothing; the sanity check's order key follows each
key type's sort order."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2206_01784_gb300 import workload  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          env=env, timeout=600, cwd=ROOT)


def test_reference_arm_line():
    out = _run(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["unit"] == line["unit"]
    assert line["config"]["workload"].startswith("256M u32 keys + u32 index values")


def test_reference_arm_other_ranks_print_nothing():
    out = _run(["--impl", "reference", "--steps", "1", "--warmup", "3"], {"RANK": "1"})
    assert out.returncode == 0 and out.stdout.strip() == ""


@pytest.mark.parametrize("kt", ["u32", "u64", "f32", "f64", "i32", "i64"])
def test_order_key_follows_sort_order(kt):
    keys = workload.keys(kt, "normal" if kt[0] == "f" else "and2", 50_000, 7)
    view = np.int64 if keys.dtype.itemsize == 8 else np.int32
    srt = oracle.sort(kt, keys)
    k = bench.order_key(torch, torch.from_numpy(srt.view(view).copy()), kt)
    assert bool((k[1:] >= k[:-1]).all())
    k2 = bench.order_key(torch, torch.from_numpy(keys.view(view).copy()), kt)
    assert not bool((k2[1:] >= k2[:-1]).all())


def test_workload_names():
    assert bench.workload_name(1 << 28, "uniform", 1) == "256M u32 keys + u32 index values, uniform keys (seed 1)"
    assert bench.workload_name(1 << 27, "uniform", 8, key_type="u64").startswith("128M u64 keys")
    assert bench.workload_name(1 << 20, "and2", 0, pairs=False) == "1M u32 keys only, and2 keys (seed 0)"
