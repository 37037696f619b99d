// Phase 3 of Onesweep (arXiv 2206.01784, Section 3, "Chained scan
// digit-binning kernel"; Figures 6-8): one single-pass digit-binning
// iteration, ~2n global words moved per pass.
//
// One block per tile of T = NT * IPT keys. Per tile:
//  1. tile id from a global atomic counter, so tiles run in order whatever the
//     hardware's block schedule (the look-back then always makes progress);
//  2. the tile's keys (and values) are staged into shared memory by bulk
//     copies on the TMA engine (one elected thread, an mbarrier completes);
//     the ragged last tile and unaligned inputs use plain loads;
//  3. homogeneous-tile short-circuit: if every key of the tile has the same
//     digit, ranking and local reorganisation are skipped and the tile is
//     written straight to its bin (Section 3, last paragraph of the kernel
//     description);
//  4. warp-level multi-split ranking: each warp walks its keys in 32-wide
//     batches; lanes holding the same digit are found, as in the paper, with
//     one ballot per digit bit ANDed together (on GB300 this measured 1.7x
//     faster than one __match_any_sync per key, which saturates the ADU
//     pipe); the lowest lane of each group bumps the warp's per-digit counter
//     in shared memory and the group reads the old value (Section 3, WLMS
//     paragraph);
//  5. block-wide scan of the per-warp counts: tile digit counts for the chained
//     scan and tile-relative bin starts for the local reorganisation;
//  6. thread i publishes (L, count of digit i) in the tile's status counter,
//     the keys (then the values) are reorganised into their local bins in
//     shared memory, then thread i walks the preceding tiles' counters for
//     digit i (decoupled look-back, bounded wait) and publishes
//     (G, inclusive prefix);
//  7. runs of keys (and values) are copied from the shared-memory bins to
//     their global bins, consecutive threads writing consecutive addresses.
//
// Full tiles take a branch-light path with no per-key bounds checks; only the
// ragged last tile of a pass checks every index.
#pragma once

#include "os_common.cuh"
#include "os_internal.h"

namespace onesweep {

// Tile geometries (threads per block, keys per thread, resident blocks per
// SM). Index = the `tile_config` argument of the launcher.
template <int KBITS, int CFG> struct TileShape;
template <> struct TileShape<32, 0> { static constexpr int NT = 256, IPT = 24, MINB = 3; };
template <> struct TileShape<32, 1> { static constexpr int NT = 256, IPT = 20, MINB = 3; };
template <> struct TileShape<32, 2> { static constexpr int NT = 256, IPT = 16, MINB = 4; };
template <> struct TileShape<32, 3> { static constexpr int NT = 512, IPT = 16, MINB = 2; };
template <> struct TileShape<64, 0> { static constexpr int NT = 256, IPT = 12, MINB = 3; };
template <> struct TileShape<64, 1> { static constexpr int NT = 256, IPT = 10, MINB = 3; };
template <> struct TileShape<64, 2> { static constexpr int NT = 256, IPT = 8, MINB = 4; };
template <> struct TileShape<64, 3> { static constexpr int NT = 512, IPT = 8, MINB = 2; };

// Digit-ranking variants of step 4.
constexpr int kRankBallot = 0;  // one ballot per digit bit (the paper's WLMS)
constexpr int kRankSmask = 1;   // per-warp lane masks built with shared-memory atomic OR
constexpr int kNumTileConfigs = 4;

template <int KBITS, bool PAIRS, int CFG = 0>
struct BinningConfig {
  static constexpr int NT = TileShape<KBITS, CFG>::NT;          // threads per block
  static constexpr int IPT = TileShape<KBITS, CFG>::IPT;        // keys per thread
  static constexpr int MIN_BLOCKS = TileShape<KBITS, CFG>::MINB;  // resident blocks per SM
  static constexpr int T = NT * IPT;                    // keys per tile
  static constexpr int NW = NT / 32;
  using K = typename KeyWord<KBITS>::type;
  static constexpr size_t kbuf_bytes = (size_t)T * sizeof(K);
  static constexpr size_t vbuf_bytes = PAIRS ? (size_t)T * 4 : 0;
  static constexpr size_t whist_bytes = (size_t)NW * kRadix * 8;  // [NW][256] {lane mask, count}
  static constexpr size_t small_bytes = 2 * kRadix * 4 + 64 * 4 + 2 * 8;
  static constexpr size_t smem_bytes = kbuf_bytes + vbuf_bytes + whist_bytes + small_bytes;
};

// Lanes of the warp whose digit equals this lane's (valid lanes only): one
// vote per digit bit (Section 3, WLMS), keeping the lanes that agree on it.
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, bool valid, uint32_t valid_mask) {
  uint32_t peers = valid_mask;
#pragma unroll
  for (int b = 0; b < kRadixBits; ++b) {
    const bool bit = (d >> b) & 1u;
    const uint32_t v = __ballot_sync(0xFFFFFFFFu, bit);
    peers &= bit ? v : ~v;
  }
  return valid ? peers : 0u;
}

// Float keys: FLIP bit 0 applies the sign-flip to loaded keys (first pass),
// bit 1 undoes it on stored keys (last pass).
template <int FLIP, typename K>
__device__ __forceinline__ K load_transform(K k) {
  return (FLIP & 1) ? flip_to_ordered(k) : k;
}
template <int FLIP, typename K>
__device__ __forceinline__ K store_transform(K k) {
  return (FLIP & 2) ? flip_from_ordered(k) : k;
}

template <int KBITS, bool PAIRS, int CFG, int RANK, int FLIP, bool FULL>
__device__ __forceinline__ void binning_tile(const PassArgs& a, unsigned char* smem, uint32_t tile, uint32_t count,
                                             bool bulk) {
  using C = BinningConfig<KBITS, PAIRS, CFG>;
  using K = typename C::K;
  constexpr int NT = C::NT, IPT = C::IPT, NW = C::NW;

  K* kbuf = reinterpret_cast<K*>(smem);
  uint32_t* vbuf = reinterpret_cast<uint32_t*>(smem + C::kbuf_bytes);
  // [NW][256] pairs {lane mask of the current batch, running count}
  uint32_t* whist = reinterpret_cast<uint32_t*>(smem + C::kbuf_bytes + C::vbuf_bytes);
  uint32_t* dstart = whist + 2 * NW * kRadix;  // [256] tile-local start of each digit's bin
  uint32_t* gbase = dstart + kRadix;        // [256] global index of local position 0 of each bin
  uint32_t* misc = gbase + kRadix;          // [64] scan scratch
  uint64_t* mbar = reinterpret_cast<uint64_t*>(misc + 64);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int shift = a.shift;
  const uint32_t mask = a.mask;

  // the next pass's status counters of this tile start at N
  if (a.status_clear && tid < kRadix) a.status_clear[(size_t)tile * kRadix + tid] = 0u;
  const uint32_t bin_offset = tid < kRadix ? __ldg(a.bin_offsets + tid) : 0u;
  uint32_t* status = a.status + (size_t)tile * kRadix;
  const bool publish = (int64_t)tile != a.fault_tile;

  if (bulk) {
    if (!mbar_wait_bounded(&mbar[0], 0, kBulkWaitLimit)) atomicOr(a.error, kErrTimeout);
  } else {
    __syncthreads();
  }

  // keys of this thread: warp-striped, batch i of warp w covers tile positions
  // [w*IPT*32 + i*32, +32), so batch order and lane order are input order
  K key[IPT];
  const uint32_t wbase = (uint32_t)warp * IPT * 32 + lane;
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const uint32_t idx = wbase + i * 32;
    key[i] = load_transform<FLIP>((FULL || idx < count) ? kbuf[idx] : K(0));
  }

  // 3. homogeneous-tile check
  const K first = load_transform<FLIP>(kbuf[0]);
  const uint32_t d0 = digit_of(first, shift, mask);
  bool same = true;
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const bool valid = FULL || wbase + i * 32 < count;
    same &= !valid || digit_of(key[i], shift, mask) == d0;
  }
  const bool homogeneous = __syncthreads_and(same) != 0;

  uint32_t digit_count = 0;  // thread d < 256: keys of digit d in this tile

  if (homogeneous) {
    if (PAIRS && bulk && !mbar_wait_bounded(&mbar[1], 0, kBulkWaitLimit)) atomicOr(a.error, kErrTimeout);
    if (tid < kRadix) {
      digit_count = (uint32_t)tid == d0 ? count : 0u;
      dstart[tid] = 0u;
      if (publish)
        st_relaxed_gpu(status + tid, ((tile == 0 ? kFlagGlobal : kFlagLocal) << kStatusShift) | digit_count);
    }
  } else {
    // 4. warp-level multi-split ranking; rank = keys of the same digit before
    //    this one in the warp's part of the tile
    uint2* wh = reinterpret_cast<uint2*>(whist) + warp * kRadix;
    uint32_t rank2[IPT / 2];  // two 16-bit ranks per register (ranks < T <= 2^16)
    const uint32_t lane_bit = 1u << lane;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const bool valid = FULL || wbase + i * 32 < count;
      const uint32_t d = digit_of(key[i], shift, mask);
      uint32_t peers, old;
      if (RANK == kRankSmask) {
        // every lane ORs its bit into its digit's mask word; OR commutes, so
        // the mask read back is exactly the lanes sharing the digit
        if (valid) atomicOr(&wh[d].x, lane_bit);
        __syncwarp();
        const uint2 mc = valid ? wh[d] : make_uint2(0u, 0u);
        peers = mc.x;
        old = mc.y;
      } else {
        const uint32_t valid_mask = FULL ? 0xFFFFFFFFu : __ballot_sync(0xFFFFFFFFu, valid);
        peers = digit_peers(d, valid, valid_mask);
        old = valid ? wh[d].y : 0u;
      }
      const uint32_t below = __popc(peers & lanemask_lt());
      __syncwarp();
      if (valid && below == 0) wh[d] = make_uint2(0u, old + __popc(peers));
      __syncwarp();
      const uint32_t r = old + below;
      if (i & 1)
        rank2[i / 2] |= r << 16;
      else
        rank2[i / 2] = r;
    }
    __syncthreads();

    // 5. tile digit counts, publish L, per-warp exclusive offsets
    if (tid < kRadix) {
#pragma unroll
      for (int w = 0; w < NW; ++w) digit_count += whist[2 * (w * kRadix + tid) + 1];
      if (publish)
        st_relaxed_gpu(status + tid, ((tile == 0 ? kFlagGlobal : kFlagLocal) << kStatusShift) | digit_count);
    }
    const uint32_t excl = block_exclusive_sum<NT>(tid < kRadix ? digit_count : 0u, misc);
    if (tid < kRadix) {
      uint32_t run = excl;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint32_t c = whist[2 * (w * kRadix + tid) + 1];
        whist[2 * (w * kRadix + tid) + 1] = run;
        run += c;
      }
      dstart[tid] = excl;
    }
    __syncthreads();

    // 6a. local reorganisation of the keys into shared-memory bins; for pairs
    //     the positions are kept (two 16-bit positions per register)
    uint32_t pos2[PAIRS ? IPT / 2 : 1];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const bool valid = FULL || wbase + i * 32 < count;
      const uint32_t r = (i & 1) ? (rank2[i / 2] >> 16) : (rank2[i / 2] & 0xFFFFu);
      const uint32_t p = valid ? wh[digit_of(key[i], shift, mask)].y + r : 0u;
      if (valid) kbuf[p] = key[i];
      if (PAIRS) {
        if (i & 1)
          pos2[i / 2] |= p << 16;
        else
          pos2[i / 2] = p;
      }
    }
    if (PAIRS) {
      // values: read this thread's values, wait for every read, then scatter
      if (bulk && !mbar_wait_bounded(&mbar[1], 0, kBulkWaitLimit)) atomicOr(a.error, kErrTimeout);
      uint32_t val[IPT];
#pragma unroll
      for (int i = 0; i < IPT; ++i) {
        const uint32_t idx = wbase + i * 32;
        val[i] = (FULL || idx < count) ? vbuf[idx] : 0u;
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < IPT; ++i)
        if (FULL || wbase + i * 32 < count) vbuf[(i & 1) ? (pos2[i / 2] >> 16) : (pos2[i / 2] & 0xFFFFu)] = val[i];
    }
  }

  // 6b. decoupled look-back for digit tid over the preceding tiles; the
  //     counters of up to kWindow predecessors are read per round trip
  if (tid < kRadix) {
    uint32_t exclusive = 0;
    if (tile > 0) {
      constexpr int kWindow = 4;
      int64_t k = (int64_t)tile - 1;  // nearest tile not yet accumulated
      uint32_t spins = 0;
      bool done = false;
      while (!done) {
        uint32_t s[kWindow];
#pragma unroll
        for (int w = 0; w < kWindow; ++w)
          s[w] = k - w >= 0 ? ld_relaxed_gpu(a.status + (size_t)(k - w) * kRadix + tid) : (kFlagGlobal << kStatusShift);
#pragma unroll
        for (int w = 0; w < kWindow && !done; ++w) {
          const uint32_t flag = s[w] >> kStatusShift;
          if (flag == kFlagNotReady) break;  // re-read from tile k next round
          exclusive += s[w] & kValueMask;
          --k;
          if (flag == kFlagGlobal || k < 0) done = true;
        }
        if (done) break;
        if (++spins >= a.spin_limit) {
          atomicOr(a.error, kErrTimeout);
          break;
        }
        if ((spins & 255u) == 0 && (ld_relaxed_gpu(a.error) & kErrTimeout)) break;
      }
      if (publish) st_relaxed_gpu(status + tid, (kFlagGlobal << kStatusShift) | (exclusive + digit_count));
    }
    gbase[tid] = bin_offset + exclusive - dstart[tid];
  }
  __syncthreads();

  // 7. coalesced scatter of each local bin run to its global bin
  K* keys_out = static_cast<K*>(a.keys_out);
  if (homogeneous) {
    const uint32_t g0 = gbase[d0];
#pragma unroll 4
    for (int i = 0; i < IPT; ++i) {
      const uint32_t j = i * NT + tid;
      if (FULL || j < count) {
        const K k = store_transform<FLIP>(load_transform<FLIP>(kbuf[j]));
        const uint32_t g = g0 + j;
        if (g < a.n) {
          keys_out[g] = k;
          if (PAIRS) a.vals_out[g] = vbuf[j];
        }
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const uint32_t j = i * NT + tid;
      if (FULL || j < count) {
        const K k = kbuf[j];
        const uint32_t g = gbase[digit_of(k, shift, mask)] + j;
        if (g < a.n) {
          keys_out[g] = store_transform<FLIP>(k);
          if (PAIRS) a.vals_out[g] = vbuf[j];
        }
      }
    }
  }
}

template <int KBITS, bool PAIRS, int CFG, int RANK, int FLIP>
__global__ void __launch_bounds__(BinningConfig<KBITS, PAIRS, CFG>::NT, BinningConfig<KBITS, PAIRS, CFG>::MIN_BLOCKS)
    binning_kernel(PassArgs a) {
  using C = BinningConfig<KBITS, PAIRS, CFG>;
  using K = typename C::K;
  constexpr int NT = C::NT, T = C::T, NW = C::NW;

  extern __shared__ __align__(128) unsigned char smem[];
  K* kbuf = reinterpret_cast<K*>(smem);
  uint32_t* vbuf = reinterpret_cast<uint32_t*>(smem + C::kbuf_bytes);
  uint32_t* whist = reinterpret_cast<uint32_t*>(smem + C::kbuf_bytes + C::vbuf_bytes);
  uint32_t* misc = whist + 2 * NW * kRadix + 2 * kRadix;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(misc + 64);
  const int tid = threadIdx.x;

  // 1. tile id
  if (tid == 0) {
    misc[NW + 1] = atomicAdd(a.tile_counter, 1u);
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
  }
  for (int i = tid; i < 2 * NW * kRadix; i += NT) whist[i] = 0;
  __syncthreads();
  const uint32_t tile = misc[NW + 1];
  if (tile >= a.num_tiles) return;  // only if the workspace's counters were not reset
  const uint32_t start = tile * (uint32_t)T;
  const uint32_t count = min((uint32_t)T, a.n - start);
  const bool full = count == (uint32_t)T;
  const bool bulk = a.use_bulk && full;

  // 2. stage the tile
  const K* keys_in = static_cast<const K*>(a.keys_in) + start;
  if (bulk) {
    if (tid == 0) {
      mbar_arrive_expect_tx(&mbar[0], (uint32_t)C::kbuf_bytes);
      bulk_copy_g2s(kbuf, keys_in, (uint32_t)C::kbuf_bytes, &mbar[0]);
      if (PAIRS) {
        mbar_arrive_expect_tx(&mbar[1], (uint32_t)C::vbuf_bytes);
        bulk_copy_g2s(vbuf, a.vals_in + start, (uint32_t)C::vbuf_bytes, &mbar[1]);
      }
    }
  } else {
    for (uint32_t i = tid; i < count; i += NT) kbuf[i] = keys_in[i];
    if (PAIRS)
      for (uint32_t i = tid; i < count; i += NT) vbuf[i] = a.vals_in[start + i];
  }

  if (full)
    binning_tile<KBITS, PAIRS, CFG, RANK, FLIP, true>(a, smem, tile, count, bulk);
  else
    binning_tile<KBITS, PAIRS, CFG, RANK, FLIP, false>(a, smem, tile, count, bulk);
}

template <int KBITS, bool PAIRS, int CFG, int RANK, int FLIP>
cudaError_t launch_binning_one(const PassArgs& a, cudaStream_t s) {
  using C = BinningConfig<KBITS, PAIRS, CFG>;
  static int configured_device = -1;  // one attribute call per device switch
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_device != dev) {
    cudaError_t e = cudaFuncSetAttribute(binning_kernel<KBITS, PAIRS, CFG, RANK, FLIP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_bytes);
    if (e != cudaSuccess) return e;
    configured_device = dev;
  }
  binning_kernel<KBITS, PAIRS, CFG, RANK, FLIP><<<a.num_tiles, C::NT, C::smem_bytes, s>>>(a);
  return cudaGetLastError();
}

template <int KBITS, bool PAIRS, int FLIP, int RANK>
cudaError_t launch_binning_flip_rank(const PassArgs& a, cudaStream_t s, int cfg) {
  switch (cfg) {
    case 1: return launch_binning_one<KBITS, PAIRS, 1, RANK, FLIP>(a, s);
    case 2: return launch_binning_one<KBITS, PAIRS, 2, RANK, FLIP>(a, s);
    case 3: return launch_binning_one<KBITS, PAIRS, 3, RANK, FLIP>(a, s);
    default: return launch_binning_one<KBITS, PAIRS, 0, RANK, FLIP>(a, s);
  }
}

// All tile geometries and both ranking variants for one (width, payload, flip).
template <int KBITS, bool PAIRS, int FLIP>
cudaError_t launch_binning_flip(const PassArgs& a, cudaStream_t s, int cfg, int rank) {
  return rank == kRankSmask ? launch_binning_flip_rank<KBITS, PAIRS, FLIP, kRankSmask>(a, s, cfg)
                            : launch_binning_flip_rank<KBITS, PAIRS, FLIP, kRankBallot>(a, s, cfg);
}

template <int KBITS, bool PAIRS>
uint32_t tile_keys_t(int cfg) {
  switch (cfg) {
    case 1: return BinningConfig<KBITS, PAIRS, 1>::T;
    case 2: return BinningConfig<KBITS, PAIRS, 2>::T;
    case 3: return BinningConfig<KBITS, PAIRS, 3>::T;
    default: return BinningConfig<KBITS, PAIRS, 0>::T;
  }
}

}  // namespace onesweep
