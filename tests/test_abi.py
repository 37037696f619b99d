"""The C-ABI library loads, exports every declared entry point and validates
arguments on the host (no GPU: nothing here reaches a CUDA call)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2206_01784_gb300 import onesweep as osw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"^OS_API\s+[\w\s\*]+?\b(os_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("os_sort_keys", "os_sort_pairs", "os_sort_workspace_bytes", "os_workspace_status"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = osw.load()
    out = subprocess.run(["nm", "-D", "--defined-only", osw.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(os_\w+)", out))
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in exported, name


def test_library_built_for_sm103a():
    # the compile-time architecture list of the device code (no GPU needed);
    # the GPU tests check the loaded code's binary version as well
    assert osw.os_build_info() == "cuda_arch_list=1030"


def test_workspace_sizes():
    u32 = osw.OS_KEY_U32
    assert osw.os_sort_workspace_bytes(u32, 1 << 20, 0, 0, 32) > (1 << 20) * 4
    assert osw.os_sort_workspace_bytes(u32, 1 << 20, 4, 0, 32) > osw.os_sort_workspace_bytes(u32, 1 << 20, 0, 0, 32)
    assert osw.os_sort_workspace_bytes(7, 100, 0, 0, 32) == 0       # bad key type
    assert osw.os_sort_workspace_bytes(u32, 100, 2, 0, 32) == 0     # bad value width
    assert osw.os_sort_workspace_bytes(u32, 100, 0, 0, 33) == 0     # bad bit range
    assert osw.os_sort_workspace_bytes(u32, 1 << 32, 0, 0, 32) == 0  # too large
    assert osw.os_sort_workspace_bytes(u32, (1 << 32) - 1, 4, 0, 32) > 8 * ((1 << 32) - 1)  # alternate buffers
    assert osw.os_sort_workspace_bytes(osw.OS_KEY_U64, 100, 0, 0, 64) > 0


def test_workspace_layout():
    lay = osw.os_sort_workspace_layout(osw.OS_KEY_U32, 10_000_000, 4, 0, 32)
    assert lay.num_places == 4
    assert lay.num_tiles == (10_000_000 + lay.tile_keys - 1) // lay.tile_keys
    offs = [lay.histogram_offset, lay.bin_offset_offset, lay.status_offset[0], lay.status_offset[1],
            lay.alt_keys_offset, lay.alt_values_offset]
    assert offs == sorted(offs) and all(o % 256 == 0 for o in offs)
    assert lay.status_offset[1] - lay.status_offset[0] >= lay.num_tiles * 256 * 4
    assert lay.alt_values_offset - lay.alt_keys_offset >= 10_000_000 * 4
    assert lay.total_bytes >= lay.alt_values_offset + 10_000_000 * 4
    one = osw.os_sort_workspace_layout(osw.OS_KEY_U32, 1000, 0, 0, 8)
    assert one.num_places == 1
    narrow = osw.os_sort_workspace_layout(osw.OS_KEY_U64, 1000, 0, 5, 50)
    assert narrow.num_places == 6


def test_host_validation_without_gpu():
    u32 = osw.OS_KEY_U32
    fake = 1 << 40  # never dereferenced: every call below fails validation first
    ws_bytes = osw.os_sort_workspace_bytes(u32, 1000, 0, 0, 32)
    assert osw.os_sort_keys(u32, fake, fake + 8192, 1 << 32, 0, 32, fake + 65536, 1 << 40, 0) == osw.OS_ERR_TOO_LARGE
    assert osw.os_sort_keys(u32, fake, fake + 8192, 1000, 0, 40, fake + 65536, ws_bytes, 0) == osw.OS_ERR_INVALID_ARG
    assert osw.os_sort_keys(u32, fake, fake + 8192, 1000, 9, 8, fake + 65536, ws_bytes, 0) == osw.OS_ERR_INVALID_ARG
    assert osw.os_sort_keys(9, fake, fake + 8192, 1000, 0, 32, fake + 65536, ws_bytes, 0) == osw.OS_ERR_INVALID_ARG
    assert osw.os_sort_keys(u32, fake, fake + 8192, 1000, 0, 32, fake + 65536, ws_bytes - 1, 0) == osw.OS_ERR_WORKSPACE
    assert osw.os_sort_keys(u32, fake, fake + 8192, 1000, 0, 32, None, ws_bytes, 0) == osw.OS_ERR_WORKSPACE
    # overlapping input and output
    assert osw.os_sort_keys(u32, fake, fake + 400, 1000, 0, 32, fake + 65536, ws_bytes, 0) == osw.OS_ERR_INVALID_ARG
    # misaligned keys
    assert osw.os_sort_keys(u32, fake + 2, fake + 8192, 1000, 0, 32, fake + 65536, ws_bytes, 0) == osw.OS_ERR_INVALID_ARG
    # pairs need both value pointers
    assert osw.os_sort_pairs(u32, fake, fake + 8192, None, fake + 20000, 1000, 0, 32, fake + 65536, 1 << 30,
                             0) == osw.OS_ERR_INVALID_ARG
    # n == 0 is a no-op
    assert osw.os_sort_keys(u32, None, None, 0, 0, 32, None, 0, 0) == osw.OS_OK


def test_status_strings():
    for s in range(6):
        assert osw.os_status_string(s)
    assert "2^32" in osw.os_status_string(osw.OS_ERR_TOO_LARGE)


def test_tile_configs_host_side():
    n_cfg = osw.os_num_tile_configs()
    assert n_cfg >= 1
    for kb in (32, 64):
        for vb in (0, 4):
            sizes = [osw.os_tile_config_keys(kb, vb, c) for c in range(n_cfg)]
            assert all(t >= 256 for t in sizes)
            ws = osw.os_sort_workspace_bytes(osw.OS_KEY_U32 if kb == 32 else osw.OS_KEY_U64, 1_000_000, vb, 0, kb)
            prev = osw.os_get_tile_config(kb, vb)
            for c in range(n_cfg):
                assert osw.os_set_tile_config(kb, vb, c) == osw.OS_OK
                assert osw.os_get_tile_config(kb, vb) == c
                lay = osw.os_sort_workspace_layout(osw.OS_KEY_U32 if kb == 32 else osw.OS_KEY_U64, 1_000_000, vb, 0, kb)
                assert lay.total_bytes == ws and lay.tile_keys == sizes[c]
            osw.os_set_tile_config(kb, vb, prev)
    assert osw.os_set_tile_config(32, 0, n_cfg) == osw.OS_ERR_INVALID_ARG
    assert osw.os_set_tile_config(16, 0, 0) == osw.OS_ERR_INVALID_ARG
    assert osw.os_tile_config_keys(32, 3, 0) == 0


def test_batch_workspace_and_validation():
    u32 = osw.OS_KEY_U32
    a = osw.os_sort_batch_workspace_bytes(u32, 1 << 20, 100, 4, 0, 32)
    b = osw.os_sort_batch_workspace_bytes(u32, 1 << 20, 1000, 4, 0, 32)
    assert 0 < a < b
    assert osw.os_sort_batch_workspace_bytes(u32, 1 << 31, 10, 4, 0, 32) == 0
    assert osw.os_sort_batch_workspace_bytes(u32, 100, -1, 4, 0, 32) == 0
    assert osw.os_sort_batch_workspace_bytes(9, 100, 1, 4, 0, 32) == 0
    fake = 1 << 40
    ws = osw.os_sort_batch_workspace_bytes(u32, 1000, 4, 0, 0, 32)
    # n_total == 0 or no segments: no-op before any CUDA call
    assert osw.os_sort_batch(u32, None, None, None, None, None, 0, 0, 0, 32, None, 0, 0) == osw.OS_OK
    # missing offsets, workspace too small, overlap
    assert osw.os_sort_batch(u32, fake, fake + 8192, None, None, None, 4, 1000, 0, 32, fake + 65536, ws, 0) == \
        osw.OS_ERR_INVALID_ARG
    assert osw.os_sort_batch(u32, fake, fake + 8192, None, None, fake + 20000, 4, 1000, 0, 32, fake + 65536, ws - 1,
                             0) == osw.OS_ERR_WORKSPACE
    assert osw.os_sort_batch(u32, fake, fake + 400, None, None, fake + 20000, 4, 1000, 0, 32, fake + 65536, ws, 0) == \
        osw.OS_ERR_INVALID_ARG


def test_size_buckets_and_tuning_table_roundtrip(tmp_path):
    from paper_2206_01784_gb300 import autotune

    nb = osw.os_num_size_buckets()
    assert nb == 4
    assert [osw.os_size_bucket(n) for n in (1, 65535, 65536, (1 << 20) - 1, 1 << 20, 1 << 24, 1 << 29)] == \
        [0, 0, 1, 1, 2, 3, 3]
    saved = autotune.current()
    try:
        table = {(32, 4, 1): {"cfg": 2}, (64, 0, 3): {"cfg": 5}}
        autotune.apply(table)
        assert osw.os_get_tile_config_bucket(32, 4, 1) == 2
        assert osw.os_get_tile_config_bucket(64, 0, 3) == 5
        assert osw.os_get_tile_config(64, 0) == 5  # the largest bucket
        # the tile of a sort follows its size bucket
        lay = osw.os_sort_workspace_layout(osw.OS_KEY_U32, 100_000, 4, 0, 32)
        assert lay.tile_keys == osw.os_tile_config_keys(32, 4, 2)
        p = tmp_path / "tiles.json"
        autotune.save(table, str(p), "test")
        assert autotune.load(str(p)) == table
        assert osw.os_set_tile_config_bucket(32, 4, nb, 0) == osw.OS_ERR_INVALID_ARG
        assert osw.os_get_tile_config_bucket(32, 4, -1) == -1
        # the digit width per bucket: 8 until set, 5-8 accepted
        assert osw.os_get_radix_bits_bucket(32, 0, 2) == 8
        autotune.apply({(32, 0, 2): {"cfg": 4, "radix_bits": 6}})
        assert osw.os_get_radix_bits_bucket(32, 0, 2) == 6
        for bad in (0, 4, 9):
            assert osw.os_set_radix_bits_bucket(32, 0, 2, bad) == osw.OS_ERR_INVALID_ARG
        assert osw.os_set_radix_bits_bucket(48, 0, 2, 6) == osw.OS_ERR_INVALID_ARG
        assert osw.os_get_radix_bits_bucket(32, 0, nb) == -1
        assert autotune.candidates() == [(c, 8) for c in range(osw.os_num_tile_configs())] + [(4, 5), (4, 6), (4, 7)]
    finally:
        autotune.apply(saved)
    assert osw.os_get_radix_bits_bucket(32, 0, 2) == 8


def test_host_api_validation_without_gpu():
    u32 = osw.OS_KEY_U32
    n = 1000
    dev_ws = osw.os_sort_workspace_bytes(u32, n, 4, 0, 32)
    host_ws = osw.os_sort_host_workspace_bytes(u32, n, 4, 0, 32)
    assert host_ws >= dev_ws + 4 * n * 4
    assert osw.os_sort_host_workspace_bytes(u32, n, 0, 0, 32) < host_ws
    assert osw.os_sort_host_workspace_bytes(9, n, 0, 0, 32) == 0
    assert osw.os_sort_host_workspace_bytes(u32, 1 << 32, 0, 0, 32) == 0
    fake = 1 << 40  # never dereferenced: every call below fails validation first
    hk, hko, hv, hvo, ws = fake, fake + 8192, fake + 16384, fake + 24576, fake + (1 << 20)
    assert osw.os_sort_pairs_host(u32, hk, hko, hv, hvo, 1 << 32, 0, 32, ws, 1 << 40, 0) == osw.OS_ERR_TOO_LARGE
    assert osw.os_sort_pairs_host(9, hk, hko, hv, hvo, n, 0, 32, ws, host_ws, 0) == osw.OS_ERR_INVALID_ARG
    assert osw.os_sort_pairs_host(u32, hk, hko, None, hvo, n, 0, 32, ws, host_ws, 0) == osw.OS_ERR_INVALID_ARG
    assert osw.os_sort_pairs_host(u32, hk, hk + 400, hv, hvo, n, 0, 32, ws, host_ws, 0) == osw.OS_ERR_INVALID_ARG
    assert osw.os_sort_pairs_host(u32, hk, hko, hv, hko + 40, n, 0, 32, ws, host_ws, 0) == osw.OS_ERR_INVALID_ARG
    assert osw.os_sort_pairs_host(u32, hk, hko, hv, hvo, n, 0, 32, ws, host_ws - 1, 0) == osw.OS_ERR_WORKSPACE
    assert osw.os_sort_pairs_host(u32, hk, hko, hv, hvo, n, 0, 32, None, host_ws, 0) == osw.OS_ERR_WORKSPACE
    assert osw.os_sort_pairs_host(u32, hk, hko, hv, hvo, n, 0, 32, ws + 8, host_ws, 0) == osw.OS_ERR_INVALID_ARG
    assert osw.os_sort_keys_host(u32, None, None, 0, 0, 32, None, 0, 0) == osw.OS_OK


def test_noalloc_scratch_covers_2_20_keys():
    # os_sort_noalloc's fixed 16 MiB scratch holds the workspace of a 2^20-key
    # sort of every key type, keys only or pairs (the limit its header states)
    for name, kt in osw.KEY_TYPES.items():
        bits = 64 if name in ("u64", "f64", "i64") else 32
        for vb in (0, 4):
            assert 0 < osw.os_sort_workspace_bytes(kt, 1 << 20, vb, 0, bits) <= 16 << 20, (name, vb)


def test_host_copy_mode_setting():
    # a process-wide setting read by the host-memory sorts; no GPU needed
    old = osw.os_get_host_copy_mode()
    assert old in (osw.OS_HOST_COPY_ENGINES, osw.OS_HOST_COPY_LINK)
    try:
        assert osw.os_set_host_copy_mode(osw.OS_HOST_COPY_LINK) == osw.OS_OK
        assert osw.os_get_host_copy_mode() == osw.OS_HOST_COPY_LINK
        assert osw.os_set_host_copy_mode(7) == osw.OS_ERR_INVALID_ARG
        assert osw.os_get_host_copy_mode() == osw.OS_HOST_COPY_LINK
        assert osw.os_set_host_copy_mode(osw.OS_HOST_COPY_ENGINES) == osw.OS_OK
        assert osw.os_get_host_copy_mode() == osw.OS_HOST_COPY_ENGINES
    finally:
        osw.os_set_host_copy_mode(old)
