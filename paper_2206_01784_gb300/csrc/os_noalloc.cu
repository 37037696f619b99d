// os_sort_noalloc: the sort with its scratch in static device memory, for
// callers that cannot allocate device memory (their memory belongs to another
// allocator, or a cudaMalloc would synchronize the device at a bad moment).
// Nothing here allocates: the scratch is one fixed array of this module, and
// its device address is looked up once per device.
#include <mutex>

#include "../../include/onesweep.h"
#include "os_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;  // 16 MiB, held by every device that loads the library
constexpr int kMaxDevices = 64;

// Device memory for the sort's workspace. In host code this name is only a
// stand-in for the symbol: its device address comes from
// cudaGetSymbolAddress below, once per device.
static __device__ __align__(256) unsigned char os_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on the
// first call for that device).
int scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return OS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, os_noalloc_scratch) != cudaSuccess || p == nullptr) return OS_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return OS_OK;
}

}  // namespace

extern "C" OS_API int os_sort_noalloc(int key_type, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                                      uint32_t* vals_out, uint64_t n, int begin_bit, int end_bit, void* stream,
                                      const void** scratch_out) {
  const bool pairs = vals_in != nullptr || vals_out != nullptr;
  const size_t need = os_sort_workspace_bytes(key_type, n, pairs ? 4 : 0, begin_bit, end_bit);
  if (need == 0) {
    // invalid arguments or n >= 2^32: let the regular checks name the error
    return onesweep::sort_on_workspace(key_type, keys_in, keys_out, vals_in, vals_out, n, begin_bit, end_bit,
                                       nullptr, 0, stream);
  }
  if (need > kNoAllocScratchBytes) return OS_ERR_SCRATCH_LIMIT;
  void* scratch = nullptr;
  const int rc = scratch_for_current_device(&scratch);
  if (rc != OS_OK) return rc;
  if (scratch_out) *scratch_out = scratch;
  return onesweep::sort_on_workspace(key_type, keys_in, keys_out, vals_in, vals_out, n, begin_bit, end_bit, scratch,
                                     kNoAllocScratchBytes, stream);
}
