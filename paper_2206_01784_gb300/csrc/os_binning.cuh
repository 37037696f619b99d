// Phase 3 of Onesweep (arXiv 2206.01784, Section 3, "Chained scan
// digit-binning kernel"; Figures 6-8): one single-pass digit-binning
// iteration, ~2n global words moved per pass.
//
// One block per tile of T = NT * IPT keys. Per tile:
//  1. tile id from a global atomic counter, so tiles run in order whatever the
//     hardware's block schedule (the look-back then always makes progress);
//  2. the tile's keys (and values) are staged into shared memory by bulk
//     copies on the TMA engine (one elected thread, an mbarrier completes).
//     The copy covers the 16-byte-aligned span around the tile, so tiles that
//     start anywhere (segments of a batch) still use it; plain loads are the
//     fallback when that span would leave the array;
//  3. early counts: each warp counts the digits of its part of the tile with
//     shared-memory atomics (the paper's privatised, atomically updated
//     histograms of the upfront kernel, here per warp and per tile);
//  4. thread i publishes (L, count of digit i) in the tile's status counter
//     and sends the first round of its look-back over the preceding tiles'
//     counters of digit i (Section 3, decoupled look-back); a block scan of
//     the counts gives the tile-relative bin starts. Homogeneous-tile
//     short-circuit: if every key has the same digit, ranking and local
//     reorganisation are skipped and the tile is written straight to its
//     bin (Section 3, last paragraph of the kernel description);
//  5. each warp's per-digit counters start at the local position of its
//     first key of that digit (tile bin start plus the lower warps' counts);
//  6. warp-level multi-split ranking: each warp walks its keys in 32-wide
//     batches and finds the lanes holding the same digit, either as in the
//     paper with one ballot per digit bit ANDed together, or by having every
//     lane OR its bit into a per-warp shared-memory mask word of its digit
//     (OR commutes, so the mask read back is exact whatever the order of the
//     atomics). The lowest lane of each group bumps the warp's counter of the
//     digit and the group reads the old value (Section 3, WLMS paragraph):
//     with counters that start at local positions, that is the key's place
//     in the tile's shared-memory bins, and the key is written there at once.
//     Every kRoundEvery batches the look-back's round in flight is folded in
//     and the next one sent, so its L2 round trips ride along the ranking. A
//     __match_any_sync per key measured 1.7x slower than the ballots on
//     GB300 (the match instruction saturates the ADU pipe) and is not used;
//     the values follow the keys' positions;
//  7. the look-back ends (bounded wait) and publishes (G, inclusive prefix),
//     and runs of keys (and values) are copied from the shared-memory bins to
//     their global bins, consecutive threads writing consecutive addresses.
//
// The paper's block publishes its counts after ranking; counting first
// publishes them a ranking earlier, so a tile's predecessors' counts are
// there by the time its ranking ends, and the separate reorganisation loop
// (re-reading each key's digit offset) disappears.
//
// In segmented mode (os_sort_batch) every segment is a sort of its own: its
// tiles form one look-back chain that starts at the segment's first tile, and
// it has its own bin offsets. Full tiles take a branch-light path with no
// per-key bounds checks; only a ragged tile checks every index.
#pragma once

#include "os_common.cuh"
#include "os_internal.h"

namespace onesweep {

// Tile geometries (threads per block, keys per thread, resident blocks per
// SM). Index = the geometry part of the launcher's tile configuration.
template <int KBITS, int CFG> struct TileShape;
template <> struct TileShape<32, 0> { static constexpr int NT = 256, IPT = 24, MINB = 3; };
template <> struct TileShape<32, 1> { static constexpr int NT = 256, IPT = 20, MINB = 3; };
template <> struct TileShape<32, 2> { static constexpr int NT = 256, IPT = 16, MINB = 4; };
template <> struct TileShape<64, 0> { static constexpr int NT = 256, IPT = 12, MINB = 3; };
template <> struct TileShape<64, 1> { static constexpr int NT = 256, IPT = 10, MINB = 3; };
template <> struct TileShape<64, 2> { static constexpr int NT = 256, IPT = 8, MINB = 4; };

// Digit-ranking variants of step 4. Two methods find the lanes sharing a
// digit: ballots (one per digit bit, the paper's WLMS; ALU work, insensitive
// to the key distribution) and shared-memory lane masks (every lane ORs its
// bit into its digit's mask word; shared-memory work that slows down when
// many lanes share a digit).
constexpr int kRankBallot = 0;    // ballots only
constexpr int kRankAdaptive = 1;  // hybrid, or ballots only where the pass's place is skewed
constexpr int kRankHybrid = 2;    // both methods, by batch (spreads the work over the ALU
                                  // and shared-memory pipes)

// Batches of the hybrid ranking that use lane masks: two of every three (the
// third uses ballots). Measured on GB300 against every other batch, every
// batch, one in three and one in four: this split is the fastest for 32-bit
// pairs, keys only and 64-bit pairs.
__host__ __device__ constexpr bool hybrid_uses_masks(int batch) { return batch % 3 != 0; }

template <int KBITS, bool PAIRS, int CFG = 0>
struct BinningConfig {
  static constexpr int NT = TileShape<KBITS, CFG>::NT;            // threads per block
  static constexpr int IPT = TileShape<KBITS, CFG>::IPT;          // keys per thread
  static constexpr int MIN_BLOCKS = TileShape<KBITS, CFG>::MINB;  // resident blocks per SM
  static constexpr int T = NT * IPT;                              // keys per tile
  static constexpr int NW = NT / 32;
  using K = typename KeyWord<KBITS>::type;
  // staging buffers hold a tile plus the slack of a 16-byte-aligned span
  static constexpr size_t kbuf_bytes = (size_t)T * sizeof(K) + 16;
  static constexpr size_t vbuf_bytes = PAIRS ? (size_t)T * 4 + 16 : 0;
  static constexpr size_t whist_bytes = (size_t)NW * kRadix * 8;  // [NW][256] lane masks, then [NW][256] counts
  static constexpr size_t small_bytes = 2 * kRadix * 4 + 64 * 4 + 2 * 8;
  static constexpr size_t smem_bytes = kbuf_bytes + vbuf_bytes + whist_bytes + small_bytes;
};

// Lanes of the warp whose digit equals this lane's (valid lanes only): one
// vote per digit bit (Section 3, WLMS), keeping the lanes that agree on it.
// RB: bits per digit.
template <int RB = kRadixBits>
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, bool valid, uint32_t valid_mask) {
  uint32_t peers = valid_mask;
#pragma unroll
  for (int b = 0; b < RB; ++b) {
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

// Where a tile sits: set up by the kernel's front-end, read by the body.
struct TileCtx {
  uint32_t tile;         // row of the tile in the status slabs
  uint32_t chain_first;  // first tile of its look-back chain
  uint32_t start;        // array index of the tile's first key
  uint32_t count;        // keys in the tile (0: no tile for this block)
  uint32_t koff, voff;   // staging offsets (elements) of the tile in kbuf / vbuf
  uint32_t out_base;     // array index of the chain's (segment's) first key
  uint32_t out_len;      // keys in the chain's segment
  uint32_t bulk;         // staged by bulk copies (wait on the mbarriers)
  uint32_t skewed;       // this place (of this segment) is skewed: rank with ballots only
  const uint32_t* bin_offsets;  // this place's 256 bin offsets (segment-relative)
};

// Warp-level multi-split ranking of one 32-key batch (step 4). Returns the
// key's rank among the keys of the same digit in this warp's part of the tile.
// msk / cnt: this warp's 256 lane-mask words and 256 running digit counts
// (separate 32-bit arrays, so random digits spread over all 32 banks).
template <bool FULL, int RB = kRadixBits>
__device__ __forceinline__ uint32_t wlms_rank(uint32_t* msk, uint32_t* cnt, uint32_t d, bool valid, uint32_t lane_bit,
                                              bool smask) {
  // the running count first: its shared-memory round trip overlaps the
  // search for peers (the previous batch's update is already visible)
  const uint32_t old = valid ? cnt[d] : 0u;
  uint32_t peers;
  if (smask) {
    // every lane ORs its bit into its digit's mask word; OR commutes, so the
    // mask read back is exactly the lanes sharing the digit
    if (valid) atomicOr(msk + d, lane_bit);
    __syncwarp();
    peers = valid ? msk[d] : 0u;
  } else {
    const uint32_t valid_mask = FULL ? 0xFFFFFFFFu : __ballot_sync(0xFFFFFFFFu, valid);
    peers = digit_peers<RB>(d, valid, valid_mask);
  }
  const uint32_t below = __popc(peers & lanemask_lt());
  __syncwarp();
  if (valid && below == 0) {
    if (smask) msk[d] = 0u;
    cnt[d] = old + __popc(peers);
  }
  __syncwarp();
  return old + below;
}

// Decoupled look-back of one digit in rounds: issue() reads the counters of
// up to W preceding tiles (one L2 round trip), consume() folds in what came
// back - stopping at a counter not yet published, which the next round reads
// again - until a G counter or the chain's first tile is reached, and then
// publishes this tile's (G, inclusive prefix). A round may stay in flight
// while the block does other work between issue() and consume().
//
// Beyond the paper's N/L/G protocol, a walk that has passed m preceding tiles
// but not yet reached a G counter publishes (A, m + 1, sum of the m + 1
// counts through this tile) in place of its L: a later walk that reads it adds
// the whole span's count and continues below it, instead of reading the m + 1
// tiles one by one. Each value a walk adds is the exact sum of a contiguous
// span ending where it reads, and the spans it adds are disjoint and
// adjacent, so the prefix is the paper's; a word only ever goes N -> L ->
// A... -> G, written by its own tile's walker.
template <int W>
struct Lookback {
  uint32_t s[W];       // counters of the round in flight
  uint32_t left;       // preceding tiles of the chain not yet accumulated
  uint32_t total;      // preceding tiles of the chain
  uint32_t exclusive;  // sum of the accumulated counters
  uint32_t own;        // this tile's count of the digit
  uint32_t* mine;      // this tile's counter of the digit (null: publish nothing)
  bool done;

  __device__ __forceinline__ void start(uint32_t tile, uint32_t chain_first) {
    left = tile - chain_first;
    total = left;
    exclusive = 0u;
    done = left == 0u;
  }
  // (G, exclusive + own): the inclusive prefix of the digit through this tile
  __device__ __forceinline__ void publish_global() {
    if (mine) st_relaxed_gpu(mine, (kFlagGlobal << kStatusShift) | (exclusive + own));
  }
  // (A, span, sum): this tile and the total - left predecessors passed so far
  __device__ __forceinline__ void publish_aggregate() {
    const uint32_t span = total - left + 1u;
    const uint32_t sum = exclusive + own;
    if (mine && span <= kAggMaxSpan && sum <= kAggValueMask)
      st_relaxed_gpu(mine, (kFlagAggregate << kStatusShift) | ((span - 1u) << kAggSpanShift) | sum);
  }
  // reads tiles chain_first + left - 1, chain_first + left - 2, ...
  __device__ __forceinline__ void issue(const uint32_t* status, uint32_t chain_first, int digit) {
#pragma unroll
    for (int w = 0; w < W; ++w)
      s[w] = (uint32_t)w < left ? ld_relaxed_gpu(status + (size_t)(chain_first + left - 1u - w) * kRadix + digit)
                                : (kFlagGlobal << kStatusShift);
  }
  __device__ __forceinline__ void consume() {
    const uint32_t left0 = left;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      if (done) break;
      const uint32_t flag = s[w] >> kStatusShift;
      if (flag == kFlagNotReady) break;  // read this tile again next round
      if (flag == kFlagAggregate) {
        // a whole span ending at this tile; the round's next rows lie inside it
        exclusive += s[w] & kAggValueMask;
        left -= ((s[w] >> kAggSpanShift) & (kAggMaxSpan - 1u)) + 1u;
        if (left == 0u) done = true;
        break;
      }
      exclusive += s[w] & kValueMask;
      --left;
      if (flag == kFlagGlobal || left == 0u) done = true;
    }
    if (done)
      publish_global();
    else if (left != left0)
      publish_aggregate();
  }
  // rounds until the walk ends, each waiting for its reads; a wait past the
  // poll limit records a timeout and still publishes (the successors' walks
  // then end instead of timing out one after another)
  __device__ __forceinline__ void finish(const PassArgs& a, uint32_t chain_first, int digit) {
    uint32_t spins = 0;
    while (!done) {
      issue(a.status, chain_first, digit);
      consume();
      if (done) break;
      if (++spins >= a.spin_limit) {
        atomicOr(a.error, kErrTimeout);
        break;
      }
      if ((spins & 255u) == 0 && (ld_relaxed_gpu(a.error) & kErrTimeout)) break;
    }
    if (!done) publish_global();
  }
};
constexpr int kLookbackWindow = 4;
// Tiles ahead whose keys (and values) a starting block prefetches into L2
// (measured at 2^28 keys on GB300: 48, 144 and 384 tiles ahead all shorten a
// pass by about 1 %; the tile's own staging copy then waits less).
constexpr uint32_t kPrefetchTiles = 48;
// Ranking batches between two look-back rounds: about one L2 round trip of
// ranking work, so a round's reads have come back when it is consumed.
#ifndef OS_ROUND_EVERY
#define OS_ROUND_EVERY 8
#endif
constexpr int kRoundEvery = OS_ROUND_EVERY;

template <int KBITS, bool PAIRS, int CFG, int RANK, int FLIP, bool FULL, int RB>
__device__ __forceinline__ void binning_tile(const PassArgs& a, unsigned char* smem, const TileCtx& c) {
  using C = BinningConfig<KBITS, PAIRS, CFG>;
  using K = typename C::K;
  constexpr int NT = C::NT, IPT = C::IPT, NW = C::NW;
  constexpr int R = 1 << RB;  // bins of this pass's digits (the tables keep rows of kRadix)
  static_assert(R <= kRadix && R <= NT, "one thread per digit");

  K* kt = reinterpret_cast<K*>(smem) + c.koff;
  uint32_t* vt = reinterpret_cast<uint32_t*>(smem + C::kbuf_bytes) + c.voff;
  // [NW][256] lane masks of the current batch, then [NW][256] digit counts
  // (turned into running local positions before the ranking)
  uint32_t* whist = reinterpret_cast<uint32_t*>(smem + C::kbuf_bytes + C::vbuf_bytes);
  uint32_t* wcnt = whist + NW * kRadix;
  uint32_t* dstart = whist + 2 * NW * kRadix;  // [256] tile-local start of each digit's bin
  uint32_t* gbase = dstart + kRadix;           // [256] segment index of local position 0 of each bin
  uint32_t* misc = gbase + kRadix;             // [64] scan scratch
  uint64_t* mbar = reinterpret_cast<uint64_t*>(misc + 64);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int shift = a.shift;
  const uint32_t mask = a.mask;
  const uint32_t dxor = a.digit_xor;
  const uint32_t tile = c.tile, count = c.count;

  // the next pass's status counters of this tile start at N
  if (a.status_clear && tid < kRadix)
    for (size_t row = tile; row < a.status_clear_rows; row += a.num_tiles) a.status_clear[row * kRadix + tid] = 0u;
  const uint32_t bin_offset = tid < R ? __ldg(c.bin_offsets + tid) : 0u;
  uint32_t* status = a.status + (size_t)tile * kRadix;
  const bool publish = (int64_t)tile != a.fault_tile;
  const bool chain_head = tile == c.chain_first;

  // this warp's lane masks and counts start at zero
  uint32_t* wmsk = whist + warp * kRadix;
  uint32_t* wc = wcnt + warp * kRadix;
#pragma unroll
  for (int i = lane; i < R; i += 32) {
    wmsk[i] = 0u;
    wc[i] = 0u;
  }

  if (c.bulk) {
    if (!mbar_wait_bounded(&mbar[0], 0, kBulkWaitLimit)) atomicOr(a.error, kErrTimeout);
  } else {
    __syncthreads();
  }
  __syncwarp();

  // keys of this thread: warp-striped, batch i of warp w covers tile positions
  // [w*IPT*32 + i*32, +32), so batch order and lane order are input order
  K key[IPT];
  const uint32_t wbase = (uint32_t)warp * IPT * 32 + lane;
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const uint32_t idx = wbase + i * 32;
    key[i] = load_transform<FLIP>((FULL || idx < count) ? kt[idx] : K(0));
  }

  // 3. early counts: each warp's digit histogram of its part of the tile
#pragma unroll
  for (int i = 0; i < IPT; ++i)
    if (FULL || wbase + i * 32 < count) atomicAdd(wc + digit_of(key[i], shift, mask, dxor), 1u);
  const uint32_t d0 = digit_of(load_transform<FLIP>(kt[0]), shift, mask, dxor);
  if (tid == 0) misc[NW] = 0u;  // set below by the digit that holds every key, if one does
  __syncthreads();

  // 4. tile digit counts: publish L now, and start the look-back (step 6),
  //    whose rounds then ride along the ranking; a tile whose keys share one
  //    digit skips ranking and reorganisation (homogeneous-tile short-circuit)
  uint32_t digit_count = 0;  // thread d < 256: keys of digit d in this tile
  if (tid < R) {
#pragma unroll
    for (int w = 0; w < NW; ++w) digit_count += wcnt[w * kRadix + tid];
    if (publish)
      st_relaxed_gpu(status + tid, ((chain_head ? kFlagGlobal : kFlagLocal) << kStatusShift) | digit_count);
  }
  const bool walker = tid < R && !chain_head;
  Lookback<kLookbackWindow> lb;
  bool issued = false;
  if (walker) {
    lb.start(tile, c.chain_first);
    lb.mine = publish ? status + tid : nullptr;
    lb.own = digit_count;
    lb.issue(a.status, c.chain_first, tid);
    issued = true;
  }
  // block scan of the counts (a warp scan, one barrier, the lower warps'
  // totals), which also tells whether every key has the same digit
  static_assert(NW < 64, "scan scratch");
  uint32_t incl = tid < R ? digit_count : 0u;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) misc[warp] = incl;
  if (tid < R && digit_count == count) misc[NW] = 1u;
  __syncthreads();
  const bool homogeneous = misc[NW] != 0u;

  if (homogeneous) {
    if (PAIRS && c.bulk && !mbar_wait_bounded(&mbar[1], 0, kBulkWaitLimit)) atomicOr(a.error, kErrTimeout);
    if (tid < R) dstart[tid] = 0u;
  } else {
    // 5. tile-local bin starts, and each warp's counters set to where its
    //    first key of each digit goes
    uint32_t excl = incl - (tid < R ? digit_count : 0u);
    for (int w = 0; w < NW; ++w)
      if (w < warp) excl += misc[w];
    if (tid < R) {
      uint32_t run = excl;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint32_t cw = wcnt[w * kRadix + tid];
        wcnt[w * kRadix + tid] = run;
        run += cw;
      }
      dstart[tid] = excl;
    }
    __syncthreads();

    // 6a. warp-level multi-split ranking straight to local positions: each
    //     key is written into its shared-memory bin as soon as it is ranked
    //     (every key is in registers since the barrier above); for pairs the
    //     positions are kept, two 16-bit positions per register
    uint32_t pos2[PAIRS ? IPT / 2 + 1 : 1];
    const uint32_t lane_bit = 1u << lane;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const bool valid = FULL || wbase + i * 32 < count;
      const bool smask = RANK == kRankHybrid && hybrid_uses_masks(i);
      const uint32_t p = wlms_rank<FULL, RB>(wmsk, wc, digit_of(key[i], shift, mask, dxor), valid, lane_bit, smask);
      if (valid) kt[p] = key[i];
      if (PAIRS) {
        if (i & 1)
          pos2[i / 2] |= p << 16;
        else
          pos2[i / 2] = p;
      }
      // a look-back round: fold in the last one's reads, send the next
      if (i % kRoundEvery == kRoundEvery - 1 && i + 1 < IPT && walker) {
        if (issued) lb.consume();
        issued = !lb.done;
        if (issued) lb.issue(a.status, c.chain_first, tid);
      }
    }
    if (PAIRS) {
      // values: read this thread's values, wait for every read, then scatter
      if (c.bulk && !mbar_wait_bounded(&mbar[1], 0, kBulkWaitLimit)) atomicOr(a.error, kErrTimeout);
      uint32_t val[IPT];
#pragma unroll
      for (int i = 0; i < IPT; ++i) {
        const uint32_t idx = wbase + i * 32;
        val[i] = (FULL || idx < count) ? vt[idx] : 0u;
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < IPT; ++i)
        if (FULL || wbase + i * 32 < count) vt[(i & 1) ? (pos2[i / 2] >> 16) : (pos2[i / 2] & 0xFFFFu)] = val[i];
    }
  }

  // 6b. the rest of the decoupled look-back: thread d walks back over the
  //     counters of digit d in the preceding tiles of the chain until it
  //     reaches a G counter; then it publishes (G, inclusive prefix)
  uint32_t exclusive = 0;
  if (walker) {
    if (issued) lb.consume();
    lb.finish(a, c.chain_first, tid);
    exclusive = lb.exclusive;
  }
  if (tid < R) {
    gbase[tid] = bin_offset + exclusive - dstart[tid];
    // the strip's last tile: where the next strip's keys of this digit start
    if (a.carry_out && tile == a.num_tiles - 1) a.carry_out[tid] = bin_offset + exclusive + digit_count;
  }
  __syncthreads();

  // 7. coalesced scatter of each local bin run to its global bin
  K* keys_out = static_cast<K*>(a.keys_out) + c.out_base;
  uint32_t* vals_out = PAIRS ? a.vals_out + c.out_base : nullptr;
  const uint32_t out_len = c.out_len;
  if (homogeneous) {
    const uint32_t g0 = gbase[d0];
#pragma unroll 4
    for (int i = 0; i < IPT; ++i) {
      const uint32_t j = i * NT + tid;
      if (FULL || j < count) {
        const K k = store_transform<FLIP>(load_transform<FLIP>(kt[j]));
        const uint32_t g = g0 + j;
        if (g < out_len) {
          keys_out[g] = k;
          if (PAIRS) vals_out[g] = vt[j];
        }
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const uint32_t j = i * NT + tid;
      if (FULL || j < count) {
        const K k = kt[j];
        const uint32_t g = gbase[digit_of(k, shift, mask, dxor)] + j;
        if (g < out_len) {
          keys_out[g] = store_transform<FLIP>(k);
          if (PAIRS) vals_out[g] = vt[j];
        }
      }
    }
  }
}

// Kernel front-end: tile id, where the tile sits, staging. SEG selects the
// segmented (batch) mode, where a.n is the length of the whole key array.
template <int KBITS, bool PAIRS, int CFG, int RANK, int FLIP, bool SEG, int RB = kRadixBits>
__global__ void __launch_bounds__(BinningConfig<KBITS, PAIRS, CFG>::NT, BinningConfig<KBITS, PAIRS, CFG>::MIN_BLOCKS)
    binning_kernel(PassArgs a) {
  using C = BinningConfig<KBITS, PAIRS, CFG>;
  using K = typename C::K;
  constexpr int NT = C::NT, T = C::T, NW = C::NW;
  constexpr uint32_t kKeysPer16B = 16 / sizeof(K);

  extern __shared__ __align__(128) unsigned char smem[];
  K* kbuf = reinterpret_cast<K*>(smem);
  uint32_t* vbuf = reinterpret_cast<uint32_t*>(smem + C::kbuf_bytes);
  uint32_t* whist = reinterpret_cast<uint32_t*>(smem + C::kbuf_bytes + C::vbuf_bytes);
  uint32_t* misc = whist + 2 * NW * kRadix + 2 * kRadix;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(misc + 64);
  __shared__ TileCtx s_ctx;
  const int tid = threadIdx.x;

  // 1. tile id and where the tile sits
  if (tid == 0) {
    const uint32_t tile = atomicAdd(a.tile_counter, 1u);
    TileCtx c{};
    c.tile = tile;
    if (SEG) {
      if (tile < *a.total_tiles) {
        const uint32_t seg = a.tile_seg[tile];
        const uint64_t s0 = a.seg_offsets[seg];
        const uint32_t len = (uint32_t)(a.seg_offsets[seg + 1] - s0);
        c.chain_first = a.tile_base[seg];
        const uint32_t local = (tile - c.chain_first) * (uint32_t)T;
        if (local < len) {
          c.start = (uint32_t)s0 + local;
          c.count = min((uint32_t)T, len - local);
          c.out_base = (uint32_t)s0;
          c.out_len = len;
          c.bin_offsets = a.bin_offsets + (size_t)seg * a.offsets_stride;
          if (RANK == kRankAdaptive && a.skew_flags) c.skewed = a.skew_flags[(size_t)seg * a.skew_stride];
        }
      }
    } else if (tile < a.num_tiles) {
      c.start = tile * (uint32_t)T;
      c.count = min((uint32_t)T, a.n - c.start);
      c.chain_first = 0;
      c.out_base = 0;
      c.out_len = a.out_total;
      c.bin_offsets = a.bin_offsets;
      if (RANK == kRankAdaptive && a.skew_flags) c.skewed = a.skew_flags[0];
    }
    if (c.count > 0 && a.use_bulk) {
      // the 16-byte-aligned span covering the tile, if it stays in the array
      const uint32_t ks = c.start & ~(kKeysPer16B - 1u);
      const uint32_t vs = c.start & ~3u;
      const uint32_t koff = c.start - ks, voff = c.start - vs;
      const uint32_t kbytes = ((koff + c.count) * (uint32_t)sizeof(K) + 15u) & ~15u;
      const uint32_t vbytes = ((voff + c.count) * 4u + 15u) & ~15u;
      c.bulk = (uint64_t)ks * sizeof(K) + kbytes <= (uint64_t)a.n * sizeof(K) &&
               (!PAIRS || (uint64_t)vs * 4u + vbytes <= (uint64_t)a.n * 4u);
      if (c.bulk) {
        c.koff = koff;
        c.voff = voff;
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(&mbar[0], kbytes);
        bulk_copy_g2s(kbuf, static_cast<const K*>(a.keys_in) + ks, kbytes, &mbar[0]);
        if (PAIRS) {
          mbar_arrive_expect_tx(&mbar[1], vbytes);
          bulk_copy_g2s(vbuf, a.vals_in + vs, vbytes, &mbar[1]);
        }
      }
    }
    // the tile kPrefetchTiles ahead starts well within one block lifetime:
    // bring it into L2 now, so its staging copy reads L2 instead of DRAM
    if (!SEG && a.use_bulk && tile + kPrefetchTiles < a.num_tiles &&
        (uint64_t)(tile + kPrefetchTiles + 1) * T <= a.n) {
      const size_t first = (size_t)(tile + kPrefetchTiles) * T;
      bulk_prefetch_l2(static_cast<const K*>(a.keys_in) + first, (uint32_t)(T * sizeof(K)));
      if (PAIRS) bulk_prefetch_l2(a.vals_in + first, (uint32_t)T * 4u);
    }
    s_ctx = c;
  }
  __syncthreads();
  const TileCtx c = s_ctx;
  if (c.count == 0) return;  // no tile left (or the workspace's counters were not reset)

  // 2. plain staging when the bulk copy does not apply
  if (!c.bulk) {
    const K* keys_in = static_cast<const K*>(a.keys_in) + c.start;
    for (uint32_t i = tid; i < c.count; i += NT) kbuf[i] = keys_in[i];
    if (PAIRS)
      for (uint32_t i = tid; i < c.count; i += NT) vbuf[i] = a.vals_in[c.start + i];
  }

  // adaptive ranking: one uniform branch per tile between two whole bodies
  // (ballots for a skewed place, the hybrid otherwise)
  constexpr int R0 = RANK == kRankAdaptive ? kRankHybrid : RANK;
  const bool ballots = RANK == kRankAdaptive && c.skewed;
  if (c.count == (uint32_t)T) {
    if (ballots)
      binning_tile<KBITS, PAIRS, CFG, kRankBallot, FLIP, true, RB>(a, smem, c);
    else
      binning_tile<KBITS, PAIRS, CFG, R0, FLIP, true, RB>(a, smem, c);
  } else {
    if (ballots)
      binning_tile<KBITS, PAIRS, CFG, kRankBallot, FLIP, false, RB>(a, smem, c);
    else
      binning_tile<KBITS, PAIRS, CFG, R0, FLIP, false, RB>(a, smem, c);
  }
}

}  // namespace onesweep
