// os_sort_keys_host / os_sort_pairs_host: the sort of an array held in host
// memory. Each call enqueues on the caller's stream the upload of the keys
// (and values) into device staging buffers inside the workspace, the sort of
// Section 3 on those buffers, and the download of the result into the host
// output buffers. The workspace starts with the device sort's own workspace
// (so os_workspace_status reads it as usual), followed by the staging buffers.
//
// The copies between host and device memory run either on the copy engines
// (cudaMemcpyAsync) or, in the host-link mode, as kernels that read or write
// the page-locked host buffers directly through their device mapping (on
// GB300 the host memory sits across the NVLink-C2C link). The mode is a
// process-wide setting; buffers that are pageable, unmapped or not 16-byte
// aligned always take the copy engines.
#include <cuda_runtime.h>

#include <atomic>

#include "../../include/onesweep.h"
#include "os_internal.h"

namespace {

std::atomic<int> g_host_copy_mode{OS_HOST_COPY_ENGINES};

// Copy of nvec 16-byte words between device memory and mapped host memory
// (either side may be host memory). Small blocks of at most 32 registers a
// thread, so one fits on an SM beside three binning blocks (which hold
// 61 440 of its 65 536 registers) while another call's sort runs; kLinkUnroll
// loads in flight per thread, and up to 4 blocks per SM, cover the link's
// latency.
constexpr int kLinkThreads = 128;
constexpr int kLinkUnroll = 4;

__global__ void __launch_bounds__(kLinkThreads, 16) link_copy_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                                 size_t nvec) {
  const size_t step = (size_t)kLinkThreads * kLinkUnroll;
  for (size_t base = (size_t)blockIdx.x * step + threadIdx.x; base < nvec; base += (size_t)gridDim.x * step) {
    uint4 v[kLinkUnroll];
#pragma unroll
    for (int u = 0; u < kLinkUnroll; ++u) {
      const size_t i = base + (size_t)u * kLinkThreads;
      if (i < nvec) v[u] = __ldcs(src + i);
    }
#pragma unroll
    for (int u = 0; u < kLinkUnroll; ++u) {
      const size_t i = base + (size_t)u * kLinkThreads;
      if (i < nvec) __stcs(dst + i, v[u]);
    }
  }
}

// Device address of a page-locked, mapped host byte (null otherwise).
void* mapped_host_byte(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Device address of a host range whose first and last bytes are both
// page-locked and mapped at device addresses `bytes - 1` apart (null
// otherwise: a range only partly page-locked takes the copy engines).
void* mapped_host(const void* p, size_t bytes) {
  char* first = static_cast<char*>(mapped_host_byte(p));
  if (!first) return nullptr;
  char* last = static_cast<char*>(mapped_host_byte(static_cast<const char*>(p) + bytes - 1));
  return last == first + (bytes - 1) ? first : nullptr;
}

// One host<->device copy: in the host-link mode, when the host side is
// mapped and both sides start 16-byte aligned, the kernel copies the whole
// 16-byte words and the copy engines the last bytes (fewer than 16); the copy
// engines copy everything otherwise.
cudaError_t copy_async(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  if (g_host_copy_mode.load(std::memory_order_relaxed) == OS_HOST_COPY_LINK && bytes >= 16) {
    const void* host = kind == cudaMemcpyHostToDevice ? src : dst;
    void* mapped = mapped_host(host, bytes);
    const void* from = kind == cudaMemcpyHostToDevice ? mapped : src;
    void* to = kind == cudaMemcpyHostToDevice ? dst : mapped;
    if (mapped && reinterpret_cast<uintptr_t>(from) % 16 == 0 && reinterpret_cast<uintptr_t>(to) % 16 == 0) {
      const size_t nvec = bytes / 16;
      int sms = 0, dev = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return cudaErrorInvalidValue;
      const size_t per_block = (size_t)kLinkThreads * kLinkUnroll;
      size_t grid = (nvec + per_block - 1) / per_block;
      if (grid > (size_t)sms * 4) grid = (size_t)sms * 4;
      link_copy_kernel<<<(unsigned)grid, kLinkThreads, 0, s>>>(static_cast<const uint4*>(from),
                                                              static_cast<uint4*>(to), nvec);
      const cudaError_t e = cudaGetLastError();
      const size_t done = nvec * 16;
      if (e != cudaSuccess || done == bytes) return e;
      return cudaMemcpyAsync(static_cast<char*>(dst) + done, static_cast<const char*>(src) + done, bytes - done,
                             kind, s);
    }
  }
  return cudaMemcpyAsync(dst, src, bytes, kind, s);
}

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
  if (copy_async(d_keys_in, keys_in, kbytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return OS_ERR_CUDA;
  if (pairs && copy_async(d_vals_in, vals_in, vbytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return OS_ERR_CUDA;
  const int rc = onesweep::sort_on_workspace(key_type, d_keys_in, d_keys_out, d_vals_in, d_vals_out, n, begin_bit,
                                             end_bit, ws, L.sort_bytes, stream);
  if (rc != OS_OK) return rc;
  if (copy_async(keys_out, d_keys_out, kbytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return OS_ERR_CUDA;
  if (pairs && copy_async(vals_out, d_vals_out, vbytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
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

OS_API int os_set_host_copy_mode(int mode) {
  if (mode != OS_HOST_COPY_ENGINES && mode != OS_HOST_COPY_LINK) return OS_ERR_INVALID_ARG;
  g_host_copy_mode.store(mode, std::memory_order_relaxed);
  return OS_OK;
}

OS_API int os_get_host_copy_mode(void) { return g_host_copy_mode.load(std::memory_order_relaxed); }

OS_API int os_sort_pairs_host(int key_type, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                              uint32_t* vals_out, uint64_t n, int begin_bit, int end_bit, void* ws, size_t ws_bytes,
                              void* stream) {
  if (!vals_in || !vals_out) return OS_ERR_INVALID_ARG;
  return sort_host(key_type, keys_in, keys_out, vals_in, vals_out, n, begin_bit, end_bit, ws, ws_bytes, stream);
}

}  // extern "C"
