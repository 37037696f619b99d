// Phase 1 and 2 of Onesweep (arXiv 2206.01784, Section 3, "Upfront histogram
// kernel" and "Exclusive sum kernel"; Figure 5).
//
// A grid sized to the SM count walks the keys tile-cyclically with 128-bit
// streaming loads. Each block keeps private per-place digit histograms in
// shared memory, updated by shared-memory atomics, and adds them to the
// global histograms with global atomics when done. The block that finishes
// last then takes the exclusive prefix sum of every place's histogram,
// producing the global bin offsets: the paper's separate exclusive-sum kernel
// is folded into the histogram kernel's last block (one launch fewer).
//
// Skewed keys (low-entropy bands, all-equal keys) make many lanes hit one
// shared counter. Each thread therefore first merges runs of equal digits
// among its own keys and issues one atomic per run.
//
// On the way, the grid also zeroes the status-counter slab of the first
// binning pass, so no separate memset of it is needed.
#include "os_common.cuh"
#include "os_internal.h"

namespace onesweep {

namespace {

constexpr int kHistThreads = 512;
constexpr int kHistVec = 4;          // 16-byte loads in flight per thread per step
constexpr int kHistBlocksPerSm = 2;

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

template <int KBITS>
__global__ void __launch_bounds__(kHistThreads, kHistBlocksPerSm) histogram_kernel(HistArgs a) {
  using K = typename KeyWord<KBITS>::type;
  constexpr int P = KBITS / 8;                // most places a key can have
  constexpr int PER_VEC = 128 / KBITS;        // keys per 16-byte vector
  constexpr int KPT = kHistVec * PER_VEC;     // keys per thread per step
  __shared__ uint32_t sh[P * kRadix];
  __shared__ uint32_t scan_tmp[kHistThreads / 32 + 1];
  __shared__ uint32_t s_last;

  const int tid = threadIdx.x;
  const int p = a.num_places;
  for (int i = tid; i < P * kRadix; i += kHistThreads) sh[i] = 0;

  // zero the first pass's status slab (grid-stride, 16-byte stores)
  if (a.clear) {
    uint4* c = reinterpret_cast<uint4*>(a.clear);
    const uint64_t nv = a.clear_words / 4;
    for (uint64_t i = (uint64_t)blockIdx.x * kHistThreads + tid; i < nv; i += (uint64_t)gridDim.x * kHistThreads)
      c[i] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();

  const uint32_t last_mask = (1u << (a.end_bit - (a.begin_bit + 8 * (p - 1)))) - 1u;
  auto place_mask = [&](int pl) -> uint32_t { return pl == p - 1 ? last_mask : 0xFFu; };
  auto ordered = [&](K k) -> K { return a.flip ? flip_to_ordered(k) : k; };

  const K* keys = static_cast<const K*>(a.keys);
  const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
  uint64_t head = ((16 - (addr & 15)) & 15) / sizeof(K);
  if (head > a.n) head = a.n;
  const uint64_t nvec = (a.n - head) / PER_VEC;
  const uint64_t tail_start = head + nvec * PER_VEC;
  const uint4* vkeys = reinterpret_cast<const uint4*>(keys + head);

  const uint64_t step = (uint64_t)gridDim.x * kHistThreads * kHistVec;
  for (uint64_t base = (uint64_t)blockIdx.x * kHistThreads * kHistVec; base < nvec; base += step) {
    K k[KPT];
    if (base + (uint64_t)kHistThreads * kHistVec <= nvec) {
      uint4 v[kHistVec];
#pragma unroll
      for (int u = 0; u < kHistVec; ++u) v[u] = __ldcs(vkeys + base + (uint64_t)u * kHistThreads + tid);
#pragma unroll
      for (int u = 0; u < kHistVec; ++u) unpack<KBITS>(v[u], k + u * PER_VEC);
#pragma unroll
      for (int j = 0; j < KPT; ++j) k[j] = ordered(k[j]);
#pragma unroll
      for (int pl = 0; pl < P; ++pl) {
        if (pl < p) {
          const int shift = a.begin_bit + 8 * pl;
          const uint32_t mask = place_mask(pl);
          uint32_t* h = sh + pl * kRadix;
          uint32_t run_digit = digit_of(k[0], shift, mask), run_len = 1;
#pragma unroll
          for (int j = 1; j < KPT; ++j) {
            uint32_t d = digit_of(k[j], shift, mask);
            if (d == run_digit) {
              ++run_len;
            } else {
              atomicAdd(h + run_digit, run_len);
              run_digit = d;
              run_len = 1;
            }
          }
          atomicAdd(h + run_digit, run_len);
        }
      }
    } else {
      // last, partial step: one key at a time
      for (int u = 0; u < kHistVec; ++u) {
        const uint64_t idx = base + (uint64_t)u * kHistThreads + tid;
        if (idx < nvec) {
          K kk[PER_VEC];
          unpack<KBITS>(__ldcs(vkeys + idx), kk);
          for (int j = 0; j < PER_VEC; ++j) {
            const K o = ordered(kk[j]);
            for (int pl = 0; pl < p; ++pl) atomicAdd(sh + pl * kRadix + digit_of(o, a.begin_bit + 8 * pl, place_mask(pl)), 1u);
          }
        }
      }
    }
  }
  // unaligned head and the tail that does not fill a vector (block 0)
  if (blockIdx.x == 0) {
    const uint64_t extra = head + (a.n - tail_start);
    if ((uint64_t)tid < extra) {
      const uint64_t i = (uint64_t)tid < head ? (uint64_t)tid : tail_start + (tid - head);
      const K o = ordered(keys[i]);
      for (int pl = 0; pl < p; ++pl) atomicAdd(sh + pl * kRadix + digit_of(o, a.begin_bit + 8 * pl, place_mask(pl)), 1u);
    }
  }
  __syncthreads();

  for (int i = tid; i < p * kRadix; i += kHistThreads) {
    const uint32_t c = sh[i];
    if (c) atomicAdd(a.hist + i, c);
  }

  // Phase 2 in the last block to finish: exclusive sum of each place's counts.
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(a.done_counter, 1u) == gridDim.x - 1) ? 1u : 0u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int pl = 0; pl < p; ++pl) {
    const uint32_t c = tid < kRadix ? ld_relaxed_gpu(a.hist + pl * kRadix + tid) : 0u;
    const uint32_t excl = block_exclusive_sum<kHistThreads>(c, scan_tmp);
    if (tid < kRadix) a.offsets[pl * kRadix + tid] = excl;
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_histogram(int key_bits, const HistArgs& a, int num_sms, cudaStream_t s) {
  const int per_vec = 128 / key_bits;
  const uint64_t nvec = a.n / per_vec + 1;
  const uint64_t per_block = (uint64_t)kHistThreads * kHistVec;
  uint64_t want = (nvec + per_block - 1) / per_block;
  uint64_t cap = (uint64_t)num_sms * kHistBlocksPerSm;
  // enough blocks to also zero the status slab quickly
  const uint64_t clear_blocks = (a.clear_words / 4 + kHistThreads - 1) / kHistThreads;
  if (want < clear_blocks) want = clear_blocks;
  int grid = (int)(want < cap ? want : cap);
  if (grid < 1) grid = 1;
  if (key_bits == 32)
    histogram_kernel<32><<<grid, kHistThreads, 0, s>>>(a);
  else
    histogram_kernel<64><<<grid, kHistThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace onesweep
