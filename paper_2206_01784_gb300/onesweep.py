"""Thin Python binding of the C ABI in ``include/onesweep.h`` (libonesweep.so).

The functions named ``os_*`` mirror the C entry points one to one and take
raw device pointers (ints), sizes and a ``cudaStream_t`` (int, 0 = legacy
default stream). The torch helpers below them only marshal tensors: they
allocate outputs and the workspace with torch and pass ``data_ptr()`` and the
current stream. Every step of the sort runs in the library's CUDA kernels;
there is no CPU fallback - if the library is missing this module raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libonesweep.so")

OS_KEY_U32, OS_KEY_U64, OS_KEY_F32, OS_KEY_F64, OS_KEY_I32, OS_KEY_I64 = 0, 1, 2, 3, 4, 5
OS_SORT_DESCENDING = 0x100  # OR into a key type: stable descending order
KEY_TYPES = {"u32": OS_KEY_U32, "u64": OS_KEY_U64, "f32": OS_KEY_F32, "f64": OS_KEY_F64, "i32": OS_KEY_I32,
             "i64": OS_KEY_I64}
KEY_BITS = {OS_KEY_U32: 32, OS_KEY_U64: 64, OS_KEY_F32: 32, OS_KEY_F64: 64, OS_KEY_I32: 32, OS_KEY_I64: 64}

OS_OK, OS_ERR_INVALID_ARG, OS_ERR_TOO_LARGE, OS_ERR_WORKSPACE, OS_ERR_CUDA, OS_ERR_TIMEOUT = range(6)
OS_ERR_SCRATCH_LIMIT = 6
OS_HOST_COPY_ENGINES, OS_HOST_COPY_LINK = 0, 1  # how the host-memory sorts move data


class OnesweepError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {os_status_string(status)} (status {status})")
        self.status = status


class WorkspaceLayout(ctypes.Structure):
    _fields_ = [
        ("total_bytes", ctypes.c_size_t),
        ("status_offset", ctypes.c_size_t * 2),
        ("histogram_offset", ctypes.c_size_t),
        ("bin_offset_offset", ctypes.c_size_t),
        ("alt_keys_offset", ctypes.c_size_t),
        ("alt_values_offset", ctypes.c_size_t),
        ("tile_keys", ctypes.c_uint32),
        ("num_tiles", ctypes.c_uint32),
        ("num_places", ctypes.c_uint32),
    ]


class LaunchTime(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("pass_", ctypes.c_int), ("ms", ctypes.c_float)]


class SortOptions(ctypes.Structure):
    """os_sort_options: the binning variant of one call (-1: process-wide) and
    its bits per digit place (0: the default, 8)."""
    _fields_ = [("tile_config", ctypes.c_int), ("radix_bits", ctypes.c_uint32)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libonesweep.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2206_01784_gb300.build.build()")
    lib = ctypes.CDLL(path)
    i32, u32, u64, i64, sz, vp = (ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64,
                                  ctypes.c_size_t, ctypes.c_void_p)
    lib.os_sort_workspace_bytes.restype = sz
    lib.os_sort_workspace_bytes.argtypes = [i32, u64, i32, i32, i32]
    lib.os_sort_workspace_layout.restype = i32
    lib.os_sort_workspace_layout.argtypes = [i32, u64, i32, i32, i32, ctypes.POINTER(WorkspaceLayout)]
    lib.os_sort_keys.restype = i32
    lib.os_sort_keys.argtypes = [i32, vp, vp, u64, i32, i32, vp, sz, vp]
    lib.os_sort_pairs.restype = i32
    lib.os_sort_pairs.argtypes = [i32, vp, vp, vp, vp, u64, i32, i32, vp, sz, vp]
    lib.os_sort_batch_workspace_bytes.restype = sz
    lib.os_sort_batch_workspace_bytes.argtypes = [i32, u64, i32, i32, i32, i32]
    lib.os_sort_batch.restype = i32
    lib.os_sort_batch.argtypes = [i32, vp, vp, vp, vp, vp, i32, u64, i32, i32, vp, sz, vp]
    opt = ctypes.POINTER(SortOptions)
    lib.os_sort_keys_ex.restype = i32
    lib.os_sort_keys_ex.argtypes = [i32, vp, vp, u64, i32, i32, vp, sz, vp, opt]
    lib.os_sort_pairs_ex.restype = i32
    lib.os_sort_pairs_ex.argtypes = [i32, vp, vp, vp, vp, u64, i32, i32, vp, sz, vp, opt]
    lib.os_sort_batch_ex.restype = i32
    lib.os_sort_batch_ex.argtypes = [i32, vp, vp, vp, vp, vp, i32, u64, i32, i32, vp, sz, vp, opt]
    lib.os_sort_noalloc.restype = i32
    lib.os_sort_noalloc.argtypes = [i32, vp, vp, vp, vp, u64, i32, i32, vp, ctypes.POINTER(ctypes.c_void_p)]
    lib.os_digit_histograms.restype = i32
    lib.os_digit_histograms.argtypes = [i32, vp, u64, i32, i32, vp, vp, vp, sz, vp]
    lib.os_workspace_status.restype = i32
    lib.os_workspace_status.argtypes = [vp, vp]
    lib.os_status_string.restype = ctypes.c_char_p
    lib.os_status_string.argtypes = [i32]
    lib.os_build_info.restype = ctypes.c_char_p
    lib.os_build_info.argtypes = []
    lib.os_binary_version.restype = i32
    lib.os_binary_version.argtypes = []
    lib.os_debug_set_lookback_fault.restype = None
    lib.os_debug_set_lookback_fault.argtypes = [i64, u32]
    lib.os_debug_set_strip_keys.restype = u64
    lib.os_debug_set_strip_keys.argtypes = [u64]
    lib.os_sort_host_workspace_bytes.restype = sz
    lib.os_sort_host_workspace_bytes.argtypes = [i32, u64, i32, i32, i32]
    lib.os_sort_keys_host.restype = i32
    lib.os_sort_keys_host.argtypes = [i32, vp, vp, u64, i32, i32, vp, sz, vp]
    lib.os_sort_pairs_host.restype = i32
    lib.os_sort_pairs_host.argtypes = [i32, vp, vp, vp, vp, u64, i32, i32, vp, sz, vp]
    lib.os_set_host_copy_mode.restype = i32
    lib.os_set_host_copy_mode.argtypes = [i32]
    lib.os_get_host_copy_mode.restype = i32
    lib.os_get_host_copy_mode.argtypes = []
    lib.os_num_tile_configs.restype = i32
    lib.os_num_tile_configs.argtypes = []
    lib.os_tile_config_keys.restype = i32
    lib.os_tile_config_keys.argtypes = [i32, i32, i32]
    lib.os_set_tile_config.restype = i32
    lib.os_set_tile_config.argtypes = [i32, i32, i32]
    lib.os_get_tile_config.restype = i32
    lib.os_get_tile_config.argtypes = [i32, i32]
    lib.os_num_size_buckets.restype = i32
    lib.os_num_size_buckets.argtypes = []
    lib.os_size_bucket.restype = i32
    lib.os_size_bucket.argtypes = [u64]
    lib.os_set_tile_config_bucket.restype = i32
    lib.os_set_tile_config_bucket.argtypes = [i32, i32, i32, i32]
    lib.os_get_tile_config_bucket.restype = i32
    lib.os_get_tile_config_bucket.argtypes = [i32, i32, i32]
    lib.os_set_radix_bits_bucket.restype = i32
    lib.os_set_radix_bits_bucket.argtypes = [i32, i32, i32, i32]
    lib.os_get_radix_bits_bucket.restype = i32
    lib.os_get_radix_bits_bucket.argtypes = [i32, i32, i32]
    lib.os_mlp_param_count.restype = i32
    lib.os_mlp_param_count.argtypes = [i32, i32]
    lib.os_mlp_forward.restype = i32
    lib.os_mlp_forward.argtypes = [vp, i32, i32, vp, i32, vp, vp]
    lib.os_mlp_loss_grad.restype = i32
    lib.os_mlp_loss_grad.argtypes = [vp, i32, i32, vp, vp, i32, vp, vp, vp]
    lib.os_mlp_adam_step.restype = i32
    lib.os_mlp_adam_step.argtypes = [vp, vp, vp, vp, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, i32, vp]
    lib.os_profile_start.restype = i32
    lib.os_profile_start.argtypes = [i32]
    lib.os_profile_stop.restype = i32
    lib.os_profile_stop.argtypes = [ctypes.POINTER(LaunchTime), i32, ctypes.POINTER(i32)]
    _lib = lib
    return lib


# ---------------------------------------------------------------- C ABI mirror

def os_sort_workspace_bytes(key_type: int, n: int, value_bytes: int, begin_bit: int, end_bit: int) -> int:
    return int(load().os_sort_workspace_bytes(key_type, n, value_bytes, begin_bit, end_bit))


def os_sort_workspace_layout(key_type: int, n: int, value_bytes: int, begin_bit: int, end_bit: int) -> WorkspaceLayout:
    lay = WorkspaceLayout()
    rc = load().os_sort_workspace_layout(key_type, n, value_bytes, begin_bit, end_bit, ctypes.byref(lay))
    if rc != OS_OK:
        raise OnesweepError(rc, "os_sort_workspace_layout")
    return lay


def os_sort_keys(key_type, keys_in, keys_out, n, begin_bit, end_bit, ws, ws_bytes, stream) -> int:
    return int(load().os_sort_keys(key_type, keys_in, keys_out, n, begin_bit, end_bit, ws, ws_bytes, stream))


def os_sort_pairs(key_type, keys_in, keys_out, vals_in, vals_out, n, begin_bit, end_bit, ws, ws_bytes,
                  stream) -> int:
    return int(load().os_sort_pairs(key_type, keys_in, keys_out, vals_in, vals_out, n, begin_bit, end_bit, ws,
                                    ws_bytes, stream))


def _options(tile_config, radix_bits=None):
    if tile_config is None and radix_bits is None:
        return None
    return ctypes.byref(SortOptions(-1 if tile_config is None else int(tile_config),
                                    0 if radix_bits is None else int(radix_bits)))


def os_sort_keys_ex(key_type, keys_in, keys_out, n, begin_bit, end_bit, ws, ws_bytes, stream,
                    tile_config=None, radix_bits=None) -> int:
    return int(load().os_sort_keys_ex(key_type, keys_in, keys_out, n, begin_bit, end_bit, ws, ws_bytes, stream,
                                      _options(tile_config, radix_bits)))


def os_sort_pairs_ex(key_type, keys_in, keys_out, vals_in, vals_out, n, begin_bit, end_bit, ws, ws_bytes, stream,
                     tile_config=None, radix_bits=None) -> int:
    return int(load().os_sort_pairs_ex(key_type, keys_in, keys_out, vals_in, vals_out, n, begin_bit, end_bit, ws,
                                       ws_bytes, stream, _options(tile_config, radix_bits)))


def os_sort_batch_ex(key_type, keys_in, keys_out, vals_in, vals_out, seg_offsets, num_segments, n_total, begin_bit,
                     end_bit, ws, ws_bytes, stream, tile_config=None, radix_bits=None) -> int:
    return int(load().os_sort_batch_ex(key_type, keys_in, keys_out, vals_in, vals_out, seg_offsets, num_segments,
                                       n_total, begin_bit, end_bit, ws, ws_bytes, stream,
                                       _options(tile_config, radix_bits)))


def os_sort_batch_workspace_bytes(key_type: int, n_total: int, num_segments: int, value_bytes: int, begin_bit: int,
                                  end_bit: int) -> int:
    return int(load().os_sort_batch_workspace_bytes(key_type, n_total, num_segments, value_bytes, begin_bit, end_bit))


def os_sort_batch(key_type, keys_in, keys_out, vals_in, vals_out, seg_offsets, num_segments, n_total, begin_bit,
                  end_bit, ws, ws_bytes, stream) -> int:
    return int(load().os_sort_batch(key_type, keys_in, keys_out, vals_in, vals_out, seg_offsets, num_segments,
                                    n_total, begin_bit, end_bit, ws, ws_bytes, stream))


def os_sort_noalloc(key_type, keys_in, keys_out, vals_in, vals_out, n, begin_bit, end_bit, stream):
    """The sort for callers that cannot allocate device memory: its scratch is
    a fixed 16 MiB of static device memory inside the library. Returns
    (status, scratch device address for os_workspace_status)."""
    scratch = ctypes.c_void_p(0)
    rc = int(load().os_sort_noalloc(key_type, keys_in, keys_out, vals_in, vals_out, n, begin_bit, end_bit, stream,
                                    ctypes.byref(scratch)))
    return rc, scratch.value


def os_digit_histograms(key_type, keys_in, n, begin_bit, end_bit, hist_out, offsets_out, ws, ws_bytes,
                        stream) -> int:
    return int(load().os_digit_histograms(key_type, keys_in, n, begin_bit, end_bit, hist_out, offsets_out, ws,
                                          ws_bytes, stream))


def os_workspace_status(ws, stream) -> int:
    return int(load().os_workspace_status(ws, stream))


def os_status_string(status: int) -> str:
    try:
        return load().os_status_string(status).decode()
    except RuntimeError:
        return f"status {status}"


def os_debug_set_lookback_fault(tile: int, spin_limit: int = 0) -> None:
    load().os_debug_set_lookback_fault(tile, spin_limit)


def os_debug_set_strip_keys(keys: int) -> int:
    return int(load().os_debug_set_strip_keys(keys))


def os_sort_host_workspace_bytes(key_type: int, n: int, value_bytes: int, begin_bit: int, end_bit: int) -> int:
    return int(load().os_sort_host_workspace_bytes(key_type, n, value_bytes, begin_bit, end_bit))


def os_sort_keys_host(key_type, keys_in, keys_out, n, begin_bit, end_bit, ws, ws_bytes, stream) -> int:
    return int(load().os_sort_keys_host(key_type, keys_in, keys_out, n, begin_bit, end_bit, ws, ws_bytes, stream))


def os_sort_pairs_host(key_type, keys_in, keys_out, vals_in, vals_out, n, begin_bit, end_bit, ws, ws_bytes,
                       stream) -> int:
    return int(load().os_sort_pairs_host(key_type, keys_in, keys_out, vals_in, vals_out, n, begin_bit, end_bit, ws,
                                         ws_bytes, stream))


def os_set_host_copy_mode(mode: int) -> int:
    return int(load().os_set_host_copy_mode(mode))


def os_get_host_copy_mode() -> int:
    return int(load().os_get_host_copy_mode())


def os_build_info() -> str:
    return load().os_build_info().decode()


def os_binary_version() -> int:
    return int(load().os_binary_version())


def os_num_tile_configs() -> int:
    return int(load().os_num_tile_configs())


def os_tile_config_keys(key_bits: int, value_bytes: int, cfg: int) -> int:
    return int(load().os_tile_config_keys(key_bits, value_bytes, cfg))


def os_set_tile_config(key_bits: int, value_bytes: int, cfg: int) -> int:
    return int(load().os_set_tile_config(key_bits, value_bytes, cfg))


def os_get_tile_config(key_bits: int, value_bytes: int) -> int:
    return int(load().os_get_tile_config(key_bits, value_bytes))


def os_num_size_buckets() -> int:
    return int(load().os_num_size_buckets())


def os_size_bucket(n: int) -> int:
    return int(load().os_size_bucket(n))


def os_set_tile_config_bucket(key_bits: int, value_bytes: int, bucket: int, cfg: int) -> int:
    return int(load().os_set_tile_config_bucket(key_bits, value_bytes, bucket, cfg))


def os_set_radix_bits_bucket(key_bits: int, value_bytes: int, bucket: int, radix_bits: int) -> int:
    return int(load().os_set_radix_bits_bucket(key_bits, value_bytes, bucket, radix_bits))


def os_get_radix_bits_bucket(key_bits: int, value_bytes: int, bucket: int) -> int:
    return int(load().os_get_radix_bits_bucket(key_bits, value_bytes, bucket))


def os_get_tile_config_bucket(key_bits: int, value_bytes: int, bucket: int) -> int:
    return int(load().os_get_tile_config_bucket(key_bits, value_bytes, bucket))


def os_mlp_param_count(features: int, hidden: int) -> int:
    return int(load().os_mlp_param_count(features, hidden))


def os_mlp_forward(params, features, hidden, x, n, y, stream) -> int:
    return int(load().os_mlp_forward(params, features, hidden, x, n, y, stream))


def os_mlp_loss_grad(params, features, hidden, x, t, n, grads, loss, stream) -> int:
    return int(load().os_mlp_loss_grad(params, features, hidden, x, t, n, grads, loss, stream))


def os_mlp_adam_step(params, grads, m, v, count, lr, beta1, beta2, eps, step, stream) -> int:
    return int(load().os_mlp_adam_step(params, grads, m, v, count, lr, beta1, beta2, eps, step, stream))


def os_profile_start(capacity: int) -> int:
    return int(load().os_profile_start(capacity))


def os_profile_stop(max_records: int = 1 << 16):
    """Returns (status, recorded launch count, [(kernel, pass, ms), ...])."""
    buf = (LaunchTime * max_records)()
    cnt = ctypes.c_int(0)
    rc = int(load().os_profile_stop(buf, max_records, ctypes.byref(cnt)))
    recs = [(buf[i].kernel, buf[i].pass_, float(buf[i].ms)) for i in range(min(cnt.value, max_records))]
    return rc, cnt.value, recs


# ---------------------------------------------------------------- torch helpers

def _torch():
    import torch
    return torch


def key_type_of(t, key_type: str | int | None = None) -> int:
    """Key type for a tensor: explicit, or by dtype (float32/64, int32/64 as
    signed, other 4/8-byte types as unsigned)."""
    torch = _torch()
    if key_type is not None:
        return KEY_TYPES[key_type] if isinstance(key_type, str) else int(key_type)
    if t.dtype == torch.float32:
        return OS_KEY_F32
    if t.dtype == torch.float64:
        return OS_KEY_F64
    if t.dtype == torch.int32:
        return OS_KEY_I32
    if t.dtype == torch.int64:
        return OS_KEY_I64
    if t.element_size() == 4:
        return OS_KEY_U32
    if t.element_size() == 8:
        return OS_KEY_U64
    raise TypeError(f"unsupported key dtype {t.dtype}")


def _stream_ptr(stream) -> int:
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def workspace(key_type: int, n: int, value_bytes: int, begin_bit: int, end_bit: int, device):
    torch = _torch()
    nbytes = os_sort_workspace_bytes(key_type, n, value_bytes, begin_bit, end_bit)
    if nbytes == 0:
        raise OnesweepError(OS_ERR_INVALID_ARG, "os_sort_workspace_bytes")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def _check(rc: int, where: str):
    if rc != OS_OK:
        raise OnesweepError(rc, where)


def _with_order(kt: int, descending: bool) -> int:
    return kt | OS_SORT_DESCENDING if descending else kt


def sort_keys(keys, begin_bit: int = 0, end_bit: int | None = None, key_type=None, out=None, ws=None,
              stream=None, descending: bool = False, radix_bits: int | None = None):
    """Stable ascending (or descending) sort of a 1-D CUDA tensor of keys;
    returns the sorted keys. radix_bits: bits per digit place (None: 8)."""
    torch = _torch()
    kt = key_type_of(keys, key_type)
    end_bit = KEY_BITS[kt] if end_bit is None else end_bit
    kt = _with_order(kt, descending)
    keys = keys.contiguous()
    n = keys.numel()
    out = torch.empty_like(keys) if out is None else out
    ws = workspace(kt, n, 0, begin_bit, end_bit, keys.device) if ws is None else ws
    _check(os_sort_keys_ex(kt, keys.data_ptr(), out.data_ptr(), n, begin_bit, end_bit, ws.data_ptr(), ws.numel(),
                           _stream_ptr(stream), radix_bits=radix_bits), "os_sort_keys")
    return out


def sort_pairs(keys, values, begin_bit: int = 0, end_bit: int | None = None, key_type=None, keys_out=None,
               values_out=None, ws=None, stream=None, descending: bool = False, radix_bits: int | None = None):
    """Stable ascending (or descending) sort of (key, uint32 value) pairs;
    returns (keys, values). radix_bits: bits per digit place (None: 8)."""
    torch = _torch()
    kt = key_type_of(keys, key_type)
    end_bit = KEY_BITS[kt] if end_bit is None else end_bit
    kt = _with_order(kt, descending)
    keys = keys.contiguous()
    values = values.contiguous()
    if values.element_size() != 4 or values.numel() != keys.numel():
        raise ValueError("values must be a 4-byte tensor with one value per key")
    n = keys.numel()
    keys_out = torch.empty_like(keys) if keys_out is None else keys_out
    values_out = torch.empty_like(values) if values_out is None else values_out
    ws = workspace(kt, n, 4, begin_bit, end_bit, keys.device) if ws is None else ws
    _check(os_sort_pairs_ex(kt, keys.data_ptr(), keys_out.data_ptr(), values.data_ptr(), values_out.data_ptr(), n,
                            begin_bit, end_bit, ws.data_ptr(), ws.numel(), _stream_ptr(stream),
                            radix_bits=radix_bits), "os_sort_pairs")
    return keys_out, values_out


def sort_host(keys, values=None, begin_bit: int = 0, end_bit: int | None = None, key_type=None, device=None,
              stream=None, descending: bool = False):
    """Stable ascending sort of keys (and uint32 values) held in host memory:
    1-D CPU tensors (pinned ones copy asynchronously) or numpy arrays. One
    os_sort_keys_host / os_sort_pairs_host call uploads, sorts on the GPU and
    downloads; returns new host arrays of the same kind once the sort is done."""
    torch = _torch()
    is_np = not isinstance(keys, torch.Tensor)
    k = torch.from_numpy(keys) if is_np else keys
    if k.device.type != "cpu":
        raise ValueError("sort_host takes host arrays; use sort_keys / sort_pairs for CUDA tensors")
    k = k.contiguous()
    kt = KEY_TYPES[key_type] if isinstance(key_type, str) else (
        int(key_type) if key_type is not None else _host_key_type(k))
    end_bit = KEY_BITS[kt] if end_bit is None else end_bit
    kt = _with_order(kt, descending)
    n = k.numel()
    ko = torch.empty_like(k, pin_memory=k.is_pinned())
    v = vo = None
    if values is not None:
        v = (torch.from_numpy(values) if is_np else values).contiguous()
        if v.element_size() != 4 or v.numel() != n:
            raise ValueError("values must be 4-byte with one value per key")
        vo = torch.empty_like(v, pin_memory=v.is_pinned())
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    nbytes = os_sort_host_workspace_bytes(kt, n, 4 if v is not None else 0, begin_bit, end_bit)
    if nbytes == 0:
        raise OnesweepError(OS_ERR_INVALID_ARG, "os_sort_host_workspace_bytes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    sp = _stream_ptr(stream)
    if v is None:
        rc = os_sort_keys_host(kt, k.data_ptr(), ko.data_ptr(), n, begin_bit, end_bit, ws.data_ptr(), nbytes, sp)
    else:
        rc = os_sort_pairs_host(kt, k.data_ptr(), ko.data_ptr(), v.data_ptr(), vo.data_ptr(), n, begin_bit, end_bit,
                                ws.data_ptr(), nbytes, sp)
    _check(rc, "os_sort_host")
    _check(os_workspace_status(ws.data_ptr(), sp), "device status")  # waits for the stream
    if is_np:
        ko = ko.numpy()
        vo = vo.numpy() if vo is not None else None
    return ko if v is None else (ko, vo)


def _host_key_type(t) -> int:
    torch = _torch()
    by_dtype = {torch.float32: OS_KEY_F32, torch.float64: OS_KEY_F64, torch.int32: OS_KEY_I32,
                torch.int64: OS_KEY_I64}
    if t.dtype in by_dtype:
        return by_dtype[t.dtype]
    if t.element_size() in (4, 8):
        return OS_KEY_U32 if t.element_size() == 4 else OS_KEY_U64
    raise TypeError(f"unsupported key dtype {t.dtype}")


def digit_histograms(keys, begin_bit: int = 0, end_bit: int | None = None, key_type=None, stream=None,
                     descending: bool = False):
    """Digit counts and global bin offsets of every place: two int32 tensors
    [p, 256] (of the complemented digits a descending sort bins by, when
    descending)."""
    torch = _torch()
    kt = key_type_of(keys, key_type)
    end_bit = KEY_BITS[kt] if end_bit is None else end_bit
    kt = _with_order(kt, descending)
    keys = keys.contiguous()
    n = keys.numel()
    p = (end_bit - begin_bit + 7) // 8
    hist = torch.empty((p, 256), dtype=torch.int32, device=keys.device)
    offs = torch.empty((p, 256), dtype=torch.int32, device=keys.device)
    ws = workspace(kt, n, 0, begin_bit, end_bit, keys.device)
    _check(os_digit_histograms(kt, keys.data_ptr(), n, begin_bit, end_bit, hist.data_ptr(), offs.data_ptr(),
                               ws.data_ptr(), ws.numel(), _stream_ptr(stream)), "os_digit_histograms")
    return hist, offs


def batch_workspace(key_type: int, n_total: int, num_segments: int, value_bytes: int, begin_bit: int, end_bit: int,
                    device):
    torch = _torch()
    nbytes = os_sort_batch_workspace_bytes(key_type, n_total, num_segments, value_bytes, begin_bit, end_bit)
    if nbytes == 0:
        raise OnesweepError(OS_ERR_INVALID_ARG, "os_sort_batch_workspace_bytes")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def sort_batch(keys, seg_offsets, values=None, begin_bit: int = 0, end_bit: int | None = None, key_type=None,
               keys_out=None, values_out=None, ws=None, stream=None, descending: bool = False):
    """Sorts each segment [seg_offsets[s], seg_offsets[s+1]) of a 1-D CUDA
    tensor on its own. seg_offsets: int64 CUDA tensor of num_segments + 1
    boundaries. Returns keys (or (keys, values))."""
    torch = _torch()
    kt = key_type_of(keys, key_type)
    end_bit = KEY_BITS[kt] if end_bit is None else end_bit
    kt = _with_order(kt, descending)
    keys = keys.contiguous()
    offs = seg_offsets.contiguous()
    if offs.dtype not in (torch.int64, torch.uint64) or offs.device != keys.device:
        raise ValueError("seg_offsets must be an int64 tensor on the keys' device")
    n = keys.numel()
    segs = offs.numel() - 1
    keys_out = torch.empty_like(keys) if keys_out is None else keys_out
    vb = 0
    vin = vout = None
    if values is not None:
        values = values.contiguous()
        if values.element_size() != 4 or values.numel() != n:
            raise ValueError("values must be a 4-byte tensor with one value per key")
        values_out = torch.empty_like(values) if values_out is None else values_out
        vb, vin, vout = 4, values.data_ptr(), values_out.data_ptr()
    ws = batch_workspace(kt, n, segs, vb, begin_bit, end_bit, keys.device) if ws is None else ws
    _check(os_sort_batch(kt, keys.data_ptr(), keys_out.data_ptr(), vin, vout, offs.data_ptr(), segs, n, begin_bit,
                         end_bit, ws.data_ptr(), ws.numel(), _stream_ptr(stream)), "os_sort_batch")
    return keys_out if values is None else (keys_out, values_out)
