// os_sort_keys_host / os_sort_pairs_host: the sort of an array held in host
// memory. Each call enqueues on the caller's stream the upload of the keys
// (and values) into device staging buffers inside the workspace, the sort of
// Section 3 on those buffers, and the download of the result into the host
// output buffers. The workspace starts with the device sort's own workspace
// (so os_workspace_status reads it as usual), followed by the staging buffers.
#include <cuda_runtime.h>

#include "../../include/onesweep.h"
#include "os_internal.h"

namespace {

constexpr size_t kAlign = 256;
size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct HostLayout {
  size_t sort_bytes = 0;  // the device sort's workspace, at offset 0
  size_t keys_in = 0, keys_out = 0, vals_in = 0, vals_out = 0;  // staging buffers
  size_t total = 0;
};

int key_bytes_of(int key_type) {
  switch (key_type & 0xFF) {  // OS_SORT_DESCENDING may be OR'd in
    case OS_KEY_U32:
    case OS_KEY_F32:
    case OS_KEY_I32: return 4;
    case OS_KEY_U64:
    case OS_KEY_F64:
    case OS_KEY_I64: return 8;
    default: return 0;
  }
}

// 0 when the arguments are invalid (the device sort's own checks then name
// the error).
size_t host_layout(int key_type, uint64_t n, int value_bytes, int begin_bit, int end_bit, HostLayout* L) {
  const size_t sort_bytes = os_sort_workspace_bytes(key_type, n, value_bytes, begin_bit, end_bit);
  const int kb = key_bytes_of(key_type);
  if (sort_bytes == 0 || kb == 0) return 0;
  const size_t kbytes = (size_t)n * kb, vbytes = (size_t)n * value_bytes;
  size_t off = round_up(sort_bytes);
  L->sort_bytes = sort_bytes;
  L->keys_in = off;
  off = round_up(off + kbytes);
  L->keys_out = off;
  off = round_up(off + kbytes);
  L->vals_in = off;
  off = round_up(off + vbytes);
  L->vals_out = off;
  off = round_up(off + vbytes);
  L->total = off;
  return off;
}

bool overlaps(const void* a, size_t abytes, const void* b, size_t bbytes) {
  if (!a || !b || abytes == 0 || bbytes == 0) return false;
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + bbytes && y < x + abytes;
}

int sort_host(int key_type, const void* keys_in, void* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
              uint64_t n, int begin_bit, int end_bit, void* ws, size_t ws_bytes, void* stream) {
  const bool pairs = vals_in != nullptr || vals_out != nullptr;
  if (pairs && (!vals_in || !vals_out)) return OS_ERR_INVALID_ARG;
  HostLayout L;
  if (host_layout(key_type, n, pairs ? 4 : 0, begin_bit, end_bit, &L) == 0) {
    // invalid key type, value width, bit range or n: the device sort names it
    return onesweep::sort_on_workspace(key_type, keys_in, keys_out, vals_in, vals_out, n, begin_bit, end_bit,
                                       nullptr, 0, stream);
  }
  if (n == 0) return OS_OK;
  if (!keys_in || !keys_out) return OS_ERR_INVALID_ARG;
  const size_t kbytes = (size_t)n * key_bytes_of(key_type), vbytes = pairs ? (size_t)n * 4 : 0;
  if (overlaps(keys_in, kbytes, keys_out, kbytes)) return OS_ERR_INVALID_ARG;
  if (pairs) {
    const void* bufs[4] = {keys_in, keys_out, vals_in, vals_out};
    const size_t sizes[4] = {kbytes, kbytes, vbytes, vbytes};
    for (int i = 0; i < 4; ++i)
      for (int j = i + 1; j < 4; ++j)
        if (overlaps(bufs[i], sizes[i], bufs[j], sizes[j])) return OS_ERR_INVALID_ARG;
  }
  if (!ws || ws_bytes < L.total) return OS_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % 16) return OS_ERR_INVALID_ARG;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  void* d_keys_in = w + L.keys_in;
  void* d_keys_out = w + L.keys_out;
  uint32_t* d_vals_in = pairs ? reinterpret_cast<uint32_t*>(w + L.vals_in) : nullptr;
  uint32_t* d_vals_out = pairs ? reinterpret_cast<uint32_t*>(w + L.vals_out) : nullptr;
  if (cudaMemcpyAsync(d_keys_in, keys_in, kbytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return OS_ERR_CUDA;
  if (pairs && cudaMemcpyAsync(d_vals_in, vals_in, vbytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return OS_ERR_CUDA;
  const int rc = onesweep::sort_on_workspace(key_type, d_keys_in, d_keys_out, d_vals_in, d_vals_out, n, begin_bit,
                                             end_bit, ws, L.sort_bytes, stream);
  if (rc != OS_OK) return rc;
  if (cudaMemcpyAsync(keys_out, d_keys_out, kbytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return OS_ERR_CUDA;
  if (pairs && cudaMemcpyAsync(vals_out, d_vals_out, vbytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return OS_ERR_CUDA;
  return OS_OK;
}

}  // namespace

extern "C" {

OS_API size_t os_sort_host_workspace_bytes(int key_type, uint64_t n, int value_bytes, int begin_bit, int end_bit) {
  HostLayout L;
  return host_layout(key_type, n, value_bytes, begin_bit, end_bit, &L);
}

OS_API int os_sort_keys_host(int key_type, const void* keys_in, void* keys_out, uint64_t n, int begin_bit,
                             int end_bit, void* ws, size_t ws_bytes, void* stream) {
  return sort_host(key_type, keys_in, keys_out, nullptr, nullptr, n, begin_bit, end_bit, ws, ws_bytes, stream);
}

OS_API int os_sort_pairs_host(int key_type, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                              uint32_t* vals_out, uint64_t n, int begin_bit, int end_bit, void* ws, size_t ws_bytes,
                              void* stream) {
  if (!vals_in || !vals_out) return OS_ERR_INVALID_ARG;
  return sort_host(key_type, keys_in, keys_out, vals_in, vals_out, n, begin_bit, end_bit, ws, ws_bytes, stream);
}

}  // extern "C"
