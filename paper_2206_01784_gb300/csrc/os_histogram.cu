// Phase 1 and 2 of Onesweep (arXiv 2206.01784, Section 3, "Upfront histogram
// kernel" and "Exclusive sum kernel"; Figure 5).
//
// A grid of one block per SM walks the keys tile-cyclically with 128-bit
// streaming loads and counts the digits of every place with shared-memory
// atomics into block-private histograms, which are added to the global
// histograms with global atomics at the end (the paper's scheme). The block
// that finishes last then takes the exclusive prefix sum of every place's
// histogram - the global bin offsets - so the paper's separate exclusive-sum
// kernel is folded into the histogram kernel's last block (one launch fewer).
//
// GB300 layout of the block-private histograms: each lane of a warp owns its
// own copy, interleaved so that lane l's counters all sit in shared-memory bank
// l (counter e of copy c at word e * kCopies + c). Every atomic of a warp then
// touches 32 distinct banks (one wavefront), and lanes never contend for one
// address, so skewed key distributions (low-entropy bands, all-equal keys) cost
// the same as uniform ones. 32-bit keys (4 places) keep 32 copies; 64-bit keys
// (8 places) keep 16 (two lanes per copy), both 128 KiB per block.
//
// On the way, the grid also zeroes the status-counter slab of the first
// binning pass, so no separate memset of it is needed.
#include "../../include/onesweep.h"
#include "os_common.cuh"
#include "os_internal.h"

namespace onesweep {

namespace {

constexpr int kHistThreads = 1024;
constexpr int kHistVec = 4;  // 16-byte loads in flight per thread per step

template <int KBITS>
struct HistLayout {
  static constexpr int P = KBITS / 8;              // places of 8-bit digits a key has
  static constexpr int kMaxP = KBITS / 5;          // most places: 5-bit digits (rounded up below)
  static constexpr int kCopies = KBITS == 32 ? 32 : 16;
  static constexpr int kEntries = P * kRadix;      // counters per copy: places x bins, for any digit width
  static constexpr size_t smem_bytes = (size_t)kEntries * kCopies * 4;
};

template <int KBITS>
__device__ __forceinline__ void unpack(const uint4& v, typename KeyWord<KBITS>::type* out);
template <>
__device__ __forceinline__ void unpack<32>(const uint4& v, uint32_t* out) {
  out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}
template <>
__device__ __forceinline__ void unpack<64>(const uint4& v, uint64_t* out) {
  out[0] = ((uint64_t)v.y << 32) | v.x;
  out[1] = ((uint64_t)v.w << 32) | v.z;
}

// FULL: the sort covers every key bit ([0, KBITS): all places 8 bits wide,
// digit i = byte i), so a digit is one shift and mask. FLIP: float keys (the
// sign-flip before counting). Both are compile-time so the counting loop, the
// kernel's whole cost (one shared-memory atomic per key and place, the issue
// slots around it), carries no per-key branches.
template <int KBITS, bool FULL, bool FLIP>
__global__ void __launch_bounds__(kHistThreads, 1) histogram_kernel(HistArgs a) {
  using K = typename KeyWord<KBITS>::type;
  using L = HistLayout<KBITS>;
  constexpr int P = L::P, C = L::kCopies;
  constexpr int PER_VEC = 128 / KBITS;     // keys per 16-byte vector
  constexpr int KPT = kHistVec * PER_VEC;  // keys per thread per step
  extern __shared__ __align__(16) uint32_t sh[];  // [P * 256][kCopies]
  __shared__ uint32_t scan_tmp[kHistThreads / 32 + 1];
  __shared__ uint32_t s_last;

  const int tid = threadIdx.x;
  const int p = a.num_places;
  {
    uint4* s4 = reinterpret_cast<uint4*>(sh);
    for (int i = tid; i < L::kEntries * C / 4; i += kHistThreads) s4[i] = make_uint4(0, 0, 0, 0);
  }

  // zero the first pass's status slab (grid-stride, 16-byte stores)
  if (a.clear) {
    uint4* c = reinterpret_cast<uint4*>(a.clear);
    const uint64_t nv = a.clear_words / 4;
    for (uint64_t i = (uint64_t)blockIdx.x * kHistThreads + tid; i < nv; i += (uint64_t)gridDim.x * kHistThreads)
      c[i] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();

  // digits of rb bits (8 in the FULL mode): place i covers bits
  // [begin + rb*i, +rb), the last one possibly narrower; counter (place,
  // digit) of this lane's copy at word ((place * 2^rb + digit) * C + copy)
  const int rb = FULL ? 8 : a.radix_bits;
  const int nbin = 1 << rb;
  const uint32_t last_mask = (1u << (a.end_bit - (a.begin_bit + rb * (p - 1)))) - 1u;
  uint32_t* mine = sh + (tid & 31) % C;
  const uint32_t top_xor = a.top_xor;
  auto count_key = [&](K k) {
    const K o = FLIP ? flip_to_ordered(k) : k;
    if (FULL) {
#pragma unroll
      for (int pl = 0; pl < P; ++pl) {
        const uint32_t d = (uint32_t)(o >> (8 * pl)) & 0xFFu;
        atomicAdd(mine + (pl * kRadix + (pl == P - 1 ? d ^ top_xor : d)) * C, 1u);
      }
    } else {
#pragma unroll
      for (int pl = 0; pl < L::kMaxP + 1; ++pl) {
        if (pl < p) {
          const uint32_t d = digit_of(o, a.begin_bit + rb * pl, pl == p - 1 ? last_mask : (uint32_t)nbin - 1u,
                                      pl == p - 1 ? top_xor : 0u);
          atomicAdd(mine + (pl * nbin + d) * C, 1u);
        }
      }
    }
  };

  const K* keys = static_cast<const K*>(a.keys);
  const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
  uint64_t head = ((16 - (addr & 15)) & 15) / sizeof(K);
  if (head > a.n) head = a.n;
  const uint64_t nvec = (a.n - head) / PER_VEC;
  const uint64_t tail_start = head + nvec * PER_VEC;
  const uint4* vkeys = reinterpret_cast<const uint4*>(keys + head);

  // full steps of kHistThreads * kHistVec vectors, the next step's loads in
  // flight while this step's keys are counted; then at most one partial step
  const uint64_t chunk = (uint64_t)kHistThreads * kHistVec;
  const uint64_t step = (uint64_t)gridDim.x * chunk;
  uint64_t base = (uint64_t)blockIdx.x * chunk;
  bool have = base + chunk <= nvec;
  uint4 v[kHistVec];
  if (have) {
#pragma unroll
    for (int u = 0; u < kHistVec; ++u) v[u] = __ldcs(vkeys + base + (uint64_t)u * kHistThreads + tid);
  }
  while (have) {
    const uint64_t next = base + step;
    const bool more = next + chunk <= nvec;
    uint4 w[kHistVec];
    if (more) {
#pragma unroll
      for (int u = 0; u < kHistVec; ++u) w[u] = __ldcs(vkeys + next + (uint64_t)u * kHistThreads + tid);
    }
    K k[KPT];
#pragma unroll
    for (int u = 0; u < kHistVec; ++u) unpack<KBITS>(v[u], k + u * PER_VEC);
#pragma unroll
    for (int j = 0; j < KPT; ++j) count_key(k[j]);
    if (more) {
#pragma unroll
      for (int u = 0; u < kHistVec; ++u) v[u] = w[u];
    }
    base = next;
    have = more;
  }
  if (base < nvec) {
    for (int u = 0; u < kHistVec; ++u) {
      const uint64_t idx = base + (uint64_t)u * kHistThreads + tid;
      if (idx < nvec) {
        K kk[PER_VEC];
        unpack<KBITS>(__ldcs(vkeys + idx), kk);
        for (int j = 0; j < PER_VEC; ++j) count_key(kk[j]);
      }
    }
  }
  // unaligned head and the tail that does not fill a vector (block 0)
  if (blockIdx.x == 0) {
    const uint64_t extra = head + (a.n - tail_start);
    if ((uint64_t)tid < extra) {
      const uint64_t i = (uint64_t)tid < head ? (uint64_t)tid : tail_start + (tid - head);
      count_key(keys[i]);
    }
  }
  __syncthreads();

  // add the block's copies of every counter (each lane starts at a different
  // copy, so a warp's reads hit distinct banks) and flush to global memory
  const int lane = tid & 31;
  for (int e = tid; e < p * nbin; e += kHistThreads) {
    uint32_t sum = 0;
#pragma unroll 8
    for (int c = 0; c < C; ++c) sum += sh[e * C + ((c + lane) % C)];
    // global histograms keep rows of kRadix words per place
    if (sum) atomicAdd(a.hist + (e >> rb) * kRadix + (e & (nbin - 1)), sum);
  }

  // Phase 2 in the last block to finish: exclusive sum of each place's counts.
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(a.done_counter, 1u) == gridDim.x - 1) ? 1u : 0u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int pl = 0; pl < p; ++pl) {
    // a descending sort bins by the complement of each digit within its
    // place: count of complemented digit t = count of digit t ^ mask
    const uint32_t pmask = pl == p - 1 ? last_mask : (uint32_t)nbin - 1u;
    const uint32_t src = a.descending ? (tid ^ pmask) : (uint32_t)tid;
    const uint32_t c = (tid < kRadix && (uint32_t)tid <= pmask) ? ld_relaxed_gpu(a.hist + pl * kRadix + src) : 0u;
    const uint32_t excl = block_exclusive_sum<kHistThreads>(c, scan_tmp);
    if (tid < kRadix) a.offsets[pl * kRadix + tid] = excl;
    // (every read of this place's counts is before the scan's barriers)
    if (a.descending && tid < kRadix) a.hist[pl * kRadix + tid] = c;
    // a place where one digit holds over 1/8 of the keys is "skewed": its
    // binning pass ranks with ballots, which do not slow down when many lanes
    // share a digit (measured on GB300: at ~10 % in one digit the lane masks
    // are still faster, at ~34 % the ballots are)
    const int skewed = __syncthreads_or(tid < kRadix && (uint64_t)c * kSkewDivisor > a.n);
    if (tid == 0 && a.skew) a.skew[pl] = skewed ? 1u : 0u;
  }
}

template <int KBITS, bool FULL, bool FLIP>
cudaError_t launch_hist_mode(const HistArgs& a, int grid, cudaStream_t s) {
  constexpr size_t bytes = HistLayout<KBITS>::smem_bytes;
  // set on every launch: an idempotent host-side attribute, so concurrent
  // callers on any device need no shared state
  cudaError_t e = cudaFuncSetAttribute(histogram_kernel<KBITS, FULL, FLIP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  histogram_kernel<KBITS, FULL, FLIP><<<grid, kHistThreads, bytes, s>>>(a);
  return cudaGetLastError();
}

template <int KBITS>
cudaError_t launch_hist_t(const HistArgs& a, int grid, cudaStream_t s) {
  const bool full = a.begin_bit == 0 && a.end_bit == KBITS && a.num_places == KBITS / 8 && a.radix_bits == 8;
  if (full) return a.flip ? launch_hist_mode<KBITS, true, true>(a, grid, s) : launch_hist_mode<KBITS, true, false>(a, grid, s);
  return a.flip ? launch_hist_mode<KBITS, false, true>(a, grid, s) : launch_hist_mode<KBITS, false, false>(a, grid, s);
}

}  // namespace

cudaError_t launch_histogram(int key_bits, const HistArgs& a, int num_sms, cudaStream_t s) {
  const int per_vec = 128 / key_bits;
  const uint64_t nvec = a.n / per_vec + 1;
  const uint64_t per_block = (uint64_t)kHistThreads * kHistVec;
  uint64_t want = (nvec + per_block - 1) / per_block;
  const uint64_t cap = (uint64_t)num_sms;  // one 1024-thread block per SM (128 KiB of shared memory)
  const uint64_t clear_blocks = (a.clear_words / 4 + kHistThreads - 1) / kHistThreads;
  if (want < clear_blocks) want = clear_blocks;
  int grid = (int)(want < cap ? want : cap);
  if (grid < 1) grid = 1;
  return key_bits == 32 ? launch_hist_t<32>(a, grid, s) : launch_hist_t<64>(a, grid, s);
}

}  // namespace onesweep

// Architecture of the device code in this library as the driver sees it
// (cudaFuncAttributes::binaryVersion of the histogram kernel, e.g. 103 for
// sm_103a), or a negative CUDA error code.
extern "C" OS_API int os_binary_version(void) {
  cudaFuncAttributes fa{};
  const cudaError_t e = cudaFuncGetAttributes(&fa, onesweep::histogram_kernel<32, true, false>);
  return e == cudaSuccess ? fa.binaryVersion : -(int)e;
}

