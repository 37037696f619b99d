// os_sort_noalloc: the sort with its scratch in static device memory, for
// callers that cannot allocate device memory (their memory belongs to another
// allocator, or a cudaMalloc would synchronize the device at a bad moment).
// Nothing here allocates: the scratch is one fixed array of this module, and
// its device address is looked up once per device and context.
#include <cuda.h>

#include <mutex>

#include "../../include/onesweep.h"
#include "os_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;  // 16 MiB, held by every device that loads the library
constexpr int kMaxDevices = 1024;

// Device memory for the sort's workspace. In host code this name is only a
// stand-in for the symbol: its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char os_noalloc_scratch[kNoAllocScratchBytes];

// The address is valid for the context it was looked up in. A device reset
// (cudaDeviceReset) or a released primary context reloads the module in a new
// context with a new address, so each device's entry remembers the id of the
// context it belongs to and is looked up again when the current one differs.
struct ScratchEntry {
  unsigned long long context_id;
  void* ptr;
};

std::mutex g_scratch_mutex;
ScratchEntry g_scratch[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Id of the current context, through the driver entry points the runtime
// hands out (no link-time dependency on the driver library).
bool current_context_id(unsigned long long* id) {
  if (!g_ctx_get_current || !g_ctx_get_id) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f)
      return false;
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f)
      return false;
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
  }
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return g_ctx_get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the scratch array on the current device, looked up with
// that device current on its first use in each context.
int scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return OS_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return OS_ERR_INVALID_ARG;
  // makes the device's primary context current (initialising it if needed)
  if (cudaSetDevice(dev) != cudaSuccess) return OS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  unsigned long long ctx_id = 0;
  if (!current_context_id(&ctx_id)) return OS_ERR_CUDA;
  ScratchEntry& e = g_scratch[dev];
  if (!e.ptr || e.context_id != ctx_id) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, os_noalloc_scratch) != cudaSuccess || p == nullptr) return OS_ERR_CUDA;
    e.ptr = p;
    e.context_id = ctx_id;
  }
  *out = e.ptr;
  return OS_OK;
}

}  // namespace

extern "C" OS_API int os_sort_noalloc(int key_type, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                                      uint32_t* vals_out, uint64_t n, int begin_bit, int end_bit, void* stream,
                                      const void** scratch_out) {
  const bool pairs = vals_in != nullptr || vals_out != nullptr;
  // argument errors first, named as by the regular entry points
  if (pairs && (vals_in == nullptr || vals_out == nullptr)) return OS_ERR_INVALID_ARG;
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
