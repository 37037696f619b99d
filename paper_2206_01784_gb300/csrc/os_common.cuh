// Device-side building blocks of the GB300 Onesweep sort (arXiv 2206.01784).
//
// Key traits (order-preserving float transform, Section 3), the chained-scan
// status counter word (Section 3, Figure 6), inline-PTX helpers for relaxed
// GPU-scope loads/stores on that word, and the mbarrier / bulk-copy (TMA
// engine, non-tensor form) primitives used to stage a tile into shared memory.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace onesweep {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;  // r = 256 bins per digit place

// Status counter (Section 3, Figure 6): two status bits over a 30-bit value.
constexpr uint32_t kStatusShift = 30;
constexpr uint32_t kValueMask = (1u << kStatusShift) - 1u;
constexpr uint32_t kFlagNotReady = 0u;  // N
constexpr uint32_t kFlagLocal = 1u;     // L: this tile's digit count
constexpr uint32_t kFlagGlobal = 2u;    // G: inclusive prefix over tiles 0..t
// A: the sum of the counts of a span of tiles ending at this one (this tile and
// the predecessors its walk has already passed), so a later walk skips the
// whole span in one read. The value then takes the low 24 bits and span - 1
// the next 6 (a span covers at most 64 tiles of at most 6144 keys).
constexpr uint32_t kFlagAggregate = 3u;
constexpr uint32_t kAggSpanShift = 24;
constexpr uint32_t kAggValueMask = (1u << kAggSpanShift) - 1u;
constexpr uint32_t kAggMaxSpan = 64;

// A digit place is skewed (its binning pass ranks with ballots only) when one
// digit holds more than 1/kSkewDivisor of the keys.
constexpr uint32_t kSkewDivisor = 8;

// Bits of the workspace's device status word.
constexpr uint32_t kErrTimeout = 1u;

// Polls of an mbarrier before a bulk copy is declared lost (each poll may
// suspend the thread for a short hardware-chosen time).
constexpr uint32_t kBulkWaitLimit = 1u << 22;

// Key word for a key width in bits.
template <int KBITS> struct KeyWord;
template <> struct KeyWord<32> { using type = uint32_t; };
template <> struct KeyWord<64> { using type = uint64_t; };

// Order-preserving ("magnitude-preserving", Section 3) map of IEEE-754 bits to
// unsigned integers: negative keys are inverted, others get the sign bit.
__device__ __forceinline__ uint32_t flip_to_ordered(uint32_t b) {
  uint32_t m = (uint32_t)((int32_t)b >> 31) | 0x80000000u;
  return b ^ m;
}
__device__ __forceinline__ uint32_t flip_from_ordered(uint32_t u) {
  uint32_t m = (uint32_t)((int32_t)(~u) >> 31) | 0x80000000u;
  return u ^ m;
}
__device__ __forceinline__ uint64_t flip_to_ordered(uint64_t b) {
  uint64_t m = (uint64_t)((int64_t)b >> 63) | 0x8000000000000000ull;
  return b ^ m;
}
__device__ __forceinline__ uint64_t flip_from_ordered(uint64_t u) {
  uint64_t m = (uint64_t)((int64_t)(~u) >> 63) | 0x8000000000000000ull;
  return u ^ m;
}

// Digit of a key at the place starting at bit `shift`, `mask` wide. For
// signed keys the top place's digit has its high bit inverted (`x`), which
// orders negative keys before non-negative ones; x = 0 otherwise.
__device__ __forceinline__ uint32_t digit_of(uint32_t u, int shift, uint32_t mask, uint32_t x = 0u) {
  return ((u >> shift) & mask) ^ x;
}
__device__ __forceinline__ uint32_t digit_of(uint64_t u, int shift, uint32_t mask, uint32_t x = 0u) {
  return ((uint32_t)(u >> shift) & mask) ^ x;
}

// ---------------------------------------------------------------- memory ops

// Relaxed GPU-scope accesses for the status counters: each word is
// self-contained (status and value travel together), so no acquire/release
// ordering is needed beyond atomicity and L2-level visibility.
__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_gpu(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// mbarrier (shared memory, CTA scope).
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of an mbarrier, at most `limit` polls. Returns
// false when the limit ran out (the caller records an error).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
  }
  return false;
}

// One bulk global->shared copy (TMA engine, untiled), completing on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Hint to bring `bytes` of global memory into L2 (no completion, no shared
// memory). src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------- block scan

// Exclusive prefix sum over the NT threads of a block (each contributes v).
// `tmp` holds NT/32 + 1 words of shared memory. Contains __syncthreads().
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_sum(uint32_t v, uint32_t* tmp, uint32_t* total = nullptr) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tmp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < NW ? tmp[lane] : 0u;
    uint32_t s = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < NW) tmp[lane] = s - w;
    if (lane == NW - 1) tmp[NW] = s;
  }
  __syncthreads();
  if (total) *total = tmp[NW];
  return tmp[warp] + x - v;
}

}  // namespace onesweep
