import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size workloads")


def read_golden(name):
    """Parse a 'key: v1 v2 ...' fixture (lines starting with # are comments)."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if ":" in line:
                k, v = line.split(":", 1)
                out[k.strip()] = [int(x) for x in v.split()]
            else:
                parts = line.split()
                out.setdefault("rows", []).append([float(x) for x in parts])
    return out


def pytest_sessionstart(session):
    """Build the oracle, the workload generator and the CUDA library in-tree
    (each is a no-op when up to date; nvcc cross-compiles without a GPU)."""
    import oracle
    from paper_2206_01784_gb300 import build as cuda_build
    from paper_2206_01784_gb300 import workload

    oracle.build()
    workload.build()
    cuda_build.build()
