// Segmented (batched) sort: many independent arrays sorted together
// (os_sort_batch). Each segment is its own Onesweep sort (arXiv 2206.01784,
// Section 3): its own digit histograms and bin offsets, its own look-back
// chain. What this file adds around the binning kernel:
//
//  * plan: one block reads the segment boundaries on the device and lays out
//    the work - each large segment's binning tiles get consecutive tile ids
//    (its look-back chain) and histogram work items; small segments are left
//    to the one-block sort. Nothing is read back to the host, so a batch can
//    be captured in a CUDA graph;
//  * per-segment histograms: work items of up to kHistChunk keys count the
//    digits of every place into their segment's histograms; the item that
//    finishes a segment last takes the exclusive sums (the segment's bin
//    offsets), as the single-array histogram kernel does for the whole array;
//  * small segments (up to one block's capacity) are sorted entirely in
//    shared memory: p in-block binning passes, one global read and one write.
#include "os_binning.cuh"
#include "os_common.cuh"
#include "os_internal.h"

namespace onesweep {

int ws_grid(uint32_t num_tiles);  // min(num_tiles, SMs of the current device)

namespace {

constexpr int kPlanThreads = 1024;
constexpr int kSegHistThreads = 1024;
constexpr int kSegHistVec = 4;  // 16-byte loads in flight per thread per step of the segment histogram

__global__ void __launch_bounds__(kPlanThreads) batch_plan_kernel(BatchArgs b) {
  __shared__ uint32_t tmp_t[kPlanThreads / 32 + 1];
  __shared__ uint32_t tmp_h[kPlanThreads / 32 + 1];
  __shared__ uint32_t s_bad;
  const int tid = threadIdx.x;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  uint32_t carry_t = 0, carry_h = 0;
  for (uint32_t base = 0; base < b.num_segments; base += kPlanThreads) {
    const uint32_t s = base + tid;
    uint32_t nt = 0, nh = 0;
    if (s < b.num_segments) {
      const uint64_t lo = b.seg_offsets[s], hi = b.seg_offsets[s + 1];
      if (hi < lo || hi > b.n_total || hi - lo >= (1ull << 30)) {
        s_bad = 1;
      } else {
        const uint32_t len = (uint32_t)(hi - lo);
        if (len > b.small_max) {
          nt = (len + b.tile_keys - 1) / b.tile_keys;
          nh = (len + b.hist_chunk - 1) / b.hist_chunk;
        }
      }
    }
    uint32_t tot_t = 0, tot_h = 0;
    const uint32_t et = block_exclusive_sum<kPlanThreads>(nt, tmp_t, &tot_t);
    const uint32_t eh = block_exclusive_sum<kPlanThreads>(nh, tmp_h, &tot_h);
    if (s < b.num_segments) {
      const uint32_t tb = carry_t + et, hb = carry_h + eh;
      b.tile_base[s] = tb;
      b.hist_base[s] = hb;
      if ((uint64_t)tb + nt <= b.max_tiles)
        for (uint32_t t = 0; t < nt; ++t) b.tile_seg[tb + t] = s;
      if ((uint64_t)hb + nh <= b.max_items)
        for (uint32_t h = 0; h < nh; ++h) b.hist_seg[hb + h] = s;
    }
    carry_t += tot_t;
    carry_h += tot_h;
    __syncthreads();
  }
  if (tid == 0) {
    b.tile_base[b.num_segments] = carry_t;
    b.hist_base[b.num_segments] = carry_h;
    const bool bad = s_bad || carry_t > b.max_tiles || carry_h > b.max_items;
    b.totals[0] = bad ? 0u : carry_t;
    b.totals[1] = bad ? 0u : carry_h;
    b.totals[2] = bad ? 1u : 0u;
    if (bad) atomicOr(b.error, kErrBadSegments);
  }
}

// Per-segment digit histograms of every place (Section 3, "Upfront histogram
// kernel", per segment). One persistent 1024-thread block per SM takes a
// contiguous range of the batch's work items (chunks of hist_chunk keys, a
// segment's items consecutive), so a block mostly meets whole runs of one
// segment's items: it counts them into block-private histograms and flushes
// them to the segment's global histograms with global atomics once per run.
// As in the single-array histogram kernel, each lane owns its own copy of the
// counters, laid out in its own shared-memory bank (counter e of copy c at
// word e * C + c), so every warp-wide atomic is one conflict-free wavefront
// and skewed keys cost no more than uniform ones; keys are read with 128-bit
// streaming loads (the unaligned head and tail of a chunk one key per
// thread). The flush that completes a segment's items takes the segment's
// exclusive sums (its bin offsets) and skewed-place flags.
template <int KBITS>
struct BatchHistLayout {
  static constexpr int P = KBITS / 8;                 // places of 8-bit digits
  static constexpr int C = KBITS == 32 ? 32 : 16;     // counter copies (lanes per copy: 32 / C)
  static constexpr size_t smem_bytes = (size_t)P * kRadix * C * 4;  // 128 KiB
};

template <int KBITS>
__global__ void __launch_bounds__(kSegHistThreads, 1) batch_histogram_kernel(BatchArgs b) {
  using K = typename KeyWord<KBITS>::type;
  using BL = BatchHistLayout<KBITS>;
  constexpr int P = BL::P, C = BL::C;
  constexpr int PER_VEC = 16 / (int)sizeof(K);  // keys per 16-byte vector
  extern __shared__ __align__(16) uint32_t sh[];  // [P * 256][C]
  __shared__ uint32_t scan_tmp[kSegHistThreads / 32 + 1];
  __shared__ uint32_t s_last;
  const int tid = threadIdx.x, lane = tid & 31;

  {
    uint4* s4 = reinterpret_cast<uint4*>(sh);
    for (int i = tid; i < P * kRadix * C / 4; i += kSegHistThreads) s4[i] = make_uint4(0, 0, 0, 0);
  }
  // zero the first pass's status slab on the way (grid-stride, 16-byte stores)
  if (b.clear) {
    uint4* c = reinterpret_cast<uint4*>(b.clear);
    const uint64_t nv = b.clear_words / 4;
    for (uint64_t i = (uint64_t)blockIdx.x * kSegHistThreads + tid; i < nv; i += (uint64_t)gridDim.x * kSegHistThreads)
      c[i] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();

  const int p = b.num_places;
  const uint32_t last_mask = (1u << (b.end_bit - (b.begin_bit + 8 * (p - 1)))) - 1u;
  const bool flip = b.flip != 0;
  uint32_t* mine = sh + (lane % C);
  auto count_key = [&](K k) {
    const K o = flip ? flip_to_ordered(k) : k;
#pragma unroll
    for (int pl = 0; pl < P; ++pl) {
      if (pl < p) {
        const uint32_t d =
            digit_of(o, b.begin_bit + 8 * pl, pl == p - 1 ? last_mask : 0xFFu, pl == p - 1 ? b.top_xor : 0u);
        atomicAdd(mine + (pl * kRadix + d) * C, 1u);
      }
    }
  };

  // add this block's copies of every counter into the segment's histograms
  // (each lane starts at a different copy, so a warp's reads and the zeroing
  // stores hit distinct banks); the flush that completes the segment's work
  // items takes its exclusive sums
  auto flush = [&](uint32_t seg, uint32_t nitems) {
    __syncthreads();
    uint32_t* gh = b.seg_hist + (size_t)seg * p * kRadix;
    for (int e = tid; e < p * kRadix; e += kSegHistThreads) {
      uint32_t sum = 0;
#pragma unroll 8
      for (int c = 0; c < C; ++c) {
        uint32_t* w = sh + e * C + ((c + lane) % C);
        sum += *w;
        *w = 0u;
      }
      if (sum) atomicAdd(gh + e, sum);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const uint32_t items = b.hist_base[seg + 1] - b.hist_base[seg];
      s_last = (atomicAdd(b.seg_done + seg, nitems) + nitems == items) ? 1u : 0u;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      const uint32_t len = (uint32_t)(b.seg_offsets[seg + 1] - b.seg_offsets[seg]);
      uint32_t* go = b.seg_bin_offsets + (size_t)seg * p * kRadix;
      for (int pl = 0; pl < p; ++pl) {
        // descending: bins of the complemented digits (count of t = count of t ^ mask)
        const uint32_t pmask = pl == p - 1 ? last_mask : 0xFFu;
        const uint32_t src = b.descending ? (tid ^ pmask) : (uint32_t)tid;
        const uint32_t c = (tid < kRadix && (uint32_t)tid <= pmask) ? ld_relaxed_gpu(gh + pl * kRadix + src) : 0u;
        const uint32_t excl = block_exclusive_sum<kSegHistThreads>(c, scan_tmp);
        if (tid < kRadix) go[pl * kRadix + tid] = excl;
        const int skewed = __syncthreads_or(tid < kRadix && (uint64_t)c * kSkewDivisor > len);
        if (tid == 0) b.seg_skew[(size_t)seg * p + pl] = skewed ? 1u : 0u;
      }
    }
    __syncthreads();
  };

  // this block's contiguous range of work items
  const uint32_t total_items = b.totals[1];
  const uint32_t per_block = (total_items + gridDim.x - 1) / gridDim.x;
  const uint32_t it0 = min(blockIdx.x * per_block, total_items);
  const uint32_t it1 = min(it0 + per_block, total_items);
  uint32_t cur = 0xFFFFFFFFu, run = 0;
  for (uint32_t item = it0; item < it1; ++item) {
    const uint32_t seg = b.hist_seg[item];
    if (seg != cur) {
      if (run) flush(cur, run);
      cur = seg;
      run = 0;
    }
    const uint64_t s0 = b.seg_offsets[seg];
    const uint32_t len = (uint32_t)(b.seg_offsets[seg + 1] - s0);
    const uint32_t lo = (item - b.hist_base[seg]) * b.hist_chunk;
    const uint32_t cnt = min(b.hist_chunk, len - lo);
    const K* keys = static_cast<const K*>(b.keys_in) + s0 + lo;
    // 16-byte vectors between an unaligned head and a tail of fewer than PER_VEC keys
    const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
    uint32_t head = (uint32_t)(((16u - (addr & 15u)) & 15u) / sizeof(K));
    if (head > cnt) head = cnt;
    const uint32_t nvec = (cnt - head) / PER_VEC;
    const uint32_t tail_start = head + nvec * PER_VEC;
    const uint4* vkeys = reinterpret_cast<const uint4*>(keys + head);
    for (uint32_t base = 0; base < nvec; base += kSegHistThreads * kSegHistVec) {
      uint4 v[kSegHistVec];
#pragma unroll
      for (int u = 0; u < kSegHistVec; ++u) {
        const uint32_t idx = base + u * kSegHistThreads + tid;
        v[u] = idx < nvec ? __ldcs(vkeys + idx) : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < kSegHistVec; ++u) {
        if (base + u * kSegHistThreads + tid < nvec) {
          const K* kk = reinterpret_cast<const K*>(&v[u]);
#pragma unroll
          for (int j = 0; j < PER_VEC; ++j) count_key(kk[j]);
        }
      }
    }
    const uint32_t extra = head + (cnt - tail_start);
    if ((uint32_t)tid < extra) count_key(keys[(uint32_t)tid < head ? tid : tail_start + (tid - head)]);
    ++run;
  }
  if (run) flush(cur, run);
}

// One-block sort of a small segment (up to LocalConfig::T keys).
template <int KBITS>
struct LocalConfig {
  static constexpr int NT = 256;
  static constexpr int IPT = KBITS == 32 ? 16 : 8;
  static constexpr int T = NT * IPT;
  static constexpr int NW = NT / 32;
};

template <int KBITS, bool PAIRS>
constexpr size_t local_smem_bytes() {
  using L = LocalConfig<KBITS>;
  return (size_t)L::T * (KBITS / 8) + (PAIRS ? (size_t)L::T * 4 : 0) + (size_t)L::NW * kRadix * 8 + 64 * 4;
}

template <int KBITS, bool PAIRS>
__global__ void __launch_bounds__(LocalConfig<KBITS>::NT) batch_local_sort_kernel(BatchArgs b) {
  using L = LocalConfig<KBITS>;
  using K = typename KeyWord<KBITS>::type;
  constexpr int NT = L::NT, IPT = L::IPT, NW = L::NW;
  extern __shared__ __align__(128) unsigned char smem[];
  K* kbuf = reinterpret_cast<K*>(smem);
  uint32_t* vbuf = reinterpret_cast<uint32_t*>(smem + (size_t)L::T * sizeof(K));
  uint32_t* whist = reinterpret_cast<uint32_t*>(smem + (size_t)L::T * sizeof(K) + (PAIRS ? (size_t)L::T * 4 : 0));
  uint32_t* misc = whist + 2 * NW * kRadix;

  const uint32_t seg = blockIdx.x;
  if (seg >= b.num_segments || b.totals[2]) return;
  const uint64_t s0 = b.seg_offsets[seg];
  const uint32_t len = (uint32_t)(b.seg_offsets[seg + 1] - s0);
  if (len == 0 || len > b.small_max || len > (uint32_t)L::T) return;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const K* kin = static_cast<const K*>(b.keys_in) + s0;
  for (uint32_t i = tid; i < len; i += NT) kbuf[i] = b.flip ? flip_to_ordered(kin[i]) : kin[i];
  if (PAIRS)
    for (uint32_t i = tid; i < len; i += NT) vbuf[i] = b.vals_in[s0 + i];

  uint32_t* wcnt = whist + NW * kRadix;
  uint32_t* wmsk = whist + warp * kRadix;
  uint32_t* wc = wcnt + warp * kRadix;
  const uint32_t wbase = (uint32_t)warp * IPT * 32 + lane;
  const uint32_t lane_bit = 1u << lane;
  for (int pass = 0; pass < b.num_places; ++pass) {
    const int shift = b.begin_bit + 8 * pass;
    const int width = min(8, b.end_bit - shift);
    const uint32_t mask = (1u << width) - 1u;
    const uint32_t dxor = (pass == b.num_places - 1 ? b.top_xor : 0u) ^ (b.descending ? mask : 0u);
    for (int i = tid; i < 2 * NW * kRadix; i += NT) whist[i] = 0;
    __syncthreads();  // staged keys (or the previous pass's scatter) visible
    K key[IPT];
    const K first = kbuf[0];
    const K digit_bits = (K)mask << shift;
    K differ = 0;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const uint32_t idx = wbase + i * 32;
      key[i] = idx < len ? kbuf[idx] : K(0);
      if (idx < len) differ |= (key[i] ^ first) & digit_bits;
    }
    if (__syncthreads_or(differ != 0) == 0) continue;  // one digit: order unchanged

    uint32_t rank[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const bool valid = wbase + i * 32 < len;
      rank[i] = wlms_rank<false>(wmsk, wc, digit_of(key[i], shift, mask, dxor), valid, lane_bit, true);
    }
    __syncthreads();
    uint32_t total = 0;
    if (tid < kRadix)
      for (int w = 0; w < NW; ++w) total += wcnt[w * kRadix + tid];
    const uint32_t excl = block_exclusive_sum<NT>(tid < kRadix ? total : 0u, misc);
    if (tid < kRadix) {
      uint32_t run = excl;
      for (int w = 0; w < NW; ++w) {
        const uint32_t cw = wcnt[w * kRadix + tid];
        wcnt[w * kRadix + tid] = run;
        run += cw;
      }
    }
    __syncthreads();
    uint32_t pos[IPT];
    uint32_t val[PAIRS ? IPT : 1];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const uint32_t idx = wbase + i * 32;
      const bool valid = idx < len;
      pos[i] = valid ? wc[digit_of(key[i], shift, mask, dxor)] + rank[i] : 0u;
      if (PAIRS) val[i] = valid ? vbuf[idx] : 0u;
    }
    __syncthreads();  // every read of the old order is done
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      if (wbase + i * 32 < len) {
        kbuf[pos[i]] = key[i];
        if (PAIRS) vbuf[pos[i]] = val[i];
      }
    }
  }
  __syncthreads();
  K* kout = static_cast<K*>(b.keys_out) + s0;
  for (uint32_t i = tid; i < len; i += NT) kout[i] = b.flip ? flip_from_ordered(kbuf[i]) : kbuf[i];
  if (PAIRS)
    for (uint32_t i = tid; i < len; i += NT) b.vals_out[s0 + i] = vbuf[i];
}

template <int KBITS, bool PAIRS>
cudaError_t launch_local(const BatchArgs& b, cudaStream_t s) {
  constexpr size_t bytes = local_smem_bytes<KBITS, PAIRS>();
  static int configured_device = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_device != dev) {
    cudaError_t e =
        cudaFuncSetAttribute(batch_local_sort_kernel<KBITS, PAIRS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    configured_device = dev;
  }
  batch_local_sort_kernel<KBITS, PAIRS><<<b.num_segments, LocalConfig<KBITS>::NT, bytes, s>>>(b);
  return cudaGetLastError();
}

}  // namespace

uint32_t batch_local_capacity(int key_bits, bool) {
  return key_bits == 32 ? LocalConfig<32>::T : LocalConfig<64>::T;
}

cudaError_t launch_batch_plan(const BatchArgs& b, cudaStream_t s) {
  batch_plan_kernel<<<1, kPlanThreads, 0, s>>>(b);
  return cudaGetLastError();
}

template <int KBITS>
cudaError_t launch_batch_histogram_t(const BatchArgs& b, int grid, cudaStream_t s) {
  constexpr size_t bytes = BatchHistLayout<KBITS>::smem_bytes;
  // set on every launch: an idempotent host-side attribute
  cudaError_t e = cudaFuncSetAttribute(batch_histogram_kernel<KBITS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return e;
  batch_histogram_kernel<KBITS><<<grid, kSegHistThreads, bytes, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_batch_histogram(int key_bits, const BatchArgs& b, cudaStream_t s) {
  // one block per SM (128 KiB of shared memory each), at most one per work item
  const int grid = ws_grid(b.max_items > 0 ? b.max_items : 1u);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  return key_bits == 32 ? launch_batch_histogram_t<32>(b, grid, s) : launch_batch_histogram_t<64>(b, grid, s);
}

cudaError_t launch_batch_local_sort(int key_bits, bool pairs, const BatchArgs& b, cudaStream_t s) {
  if (key_bits == 32) return pairs ? launch_local<32, true>(b, s) : launch_local<32, false>(b, s);
  return pairs ? launch_local<64, true>(b, s) : launch_local<64, false>(b, s);
}

}  // namespace onesweep
