// Warp-specialised, persistent form of one chained-scan digit-binning pass
// (arXiv 2206.01784, Section 3, "Chained scan digit-binning kernel";
// Figures 6-8). Same arithmetic as binning_kernel (os_binning.cuh): tile ids
// from an atomic counter, warp-level multi-split ranking, a scan of the
// per-warp digit counts, decoupled look-back over the preceding tiles' status
// counters, a shared-memory reorganisation and a coalesced scatter. What
// changes is who does each step, and when.
//
// One block per SM stays resident for the whole pass and runs two warp
// roles that hand tiles to one another through mbarriers in shared memory:
//
//   rankers (NR warps)  move the staged tile into registers, which frees the
//                       staging buffer: one ranker thread then stages the
//                       next tile there with bulk copies on the TMA engine
//                       (its tile id taken one tile ahead), so it is on its
//                       way while the current one is ranked. They rank the
//                       tile, publish each digit's (L, count), scan, and
//                       reorganise keys and values into one of two sorted
//                       buffers;
//   writers (8 warps)   for the tile in the other sorted buffer: thread d
//                       walks digit d's look-back chain and publishes
//                       (G, inclusive prefix), then the writers copy the bin
//                       runs to their global bins.
//
// So the bulk copy of tile i+1, the ranking of tile i and the look-back and
// write-out of tile i-1 overlap in every block, instead of each block waiting
// for its copy and for its look-back in turn.
//
// Progress: a block takes tile ids in increasing order and finishes them in
// that order; a tile's L counters are published before its rankers wait on
// anything that depends on a later tile, and its look-back reads only earlier
// tiles. The earliest unfinished tile therefore always progresses, whatever
// the blocks' schedule (the argument of Section 3 for the atomic tile id).
//
// Every wait is bounded: a pipeline wait that runs out, or that sees the
// device status word set by another block, makes the role stop; the block's
// other role then stops at its next wait. A role decides to stop with a
// barrier reduction over all of its threads, so its threads always take the
// same branch; a block never exits with a bulk copy still writing into its
// shared memory.
#pragma once

#include "os_binning.cuh"

namespace onesweep {

// Shapes of the persistent kernel: ranker warps, keys per ranker thread and
// writer warps (measured on GB300 at 2^28 u32 pairs: 24 rankers x 8 keys with
// 8 writers 1.415 ms per pass, 16 x 12 with 8 writers 1.434, with 16 writers
// 1.462). Shared memory holds one staging buffer and two sorted buffers of a
// tile, plus the rankers' per-warp digit tables.
template <int KBITS, bool PAIRS> struct WsShape;
template <> struct WsShape<32, true> { static constexpr int NR = 24, IPT = 8, NWR = 8; };    // 6144-key tiles
template <> struct WsShape<32, false> { static constexpr int NR = 16, IPT = 16, NWR = 8; };  // 8192-key tiles
template <> struct WsShape<64, true> { static constexpr int NR = 16, IPT = 8, NWR = 8; };    // 4096-key tiles
template <> struct WsShape<64, false> { static constexpr int NR = 16, IPT = 8, NWR = 8; };   // 4096-key tiles

// Where a tile sits (written by the staging thread for the rankers, then by the
// rankers for the writers). count == 0: no more tiles.
struct WsTile {
  uint32_t tile, start, count, bulk, koff, voff, pad0, pad1;
};

template <int KBITS, bool PAIRS>
struct WsConfig {
  using K = typename KeyWord<KBITS>::type;
  static constexpr int NR = WsShape<KBITS, PAIRS>::NR;    // ranker warps
  static constexpr int IPT = WsShape<KBITS, PAIRS>::IPT;  // keys per ranker thread
  static constexpr int NWR = WsShape<KBITS, PAIRS>::NWR;  // writer warps; the first 8 walk digit d's chain
  static_assert(NWR * 32 >= kRadix, "one look-back walker per digit");
  static constexpr int NRT = NR * 32, NWT = NWR * 32;
  static constexpr int NT = NRT + NWT;
  static constexpr int T = NRT * IPT;                     // keys per tile
  static constexpr uint32_t kVB = PAIRS ? 4u : 0u;
  // 32-bit keys with values: the sorted buffers hold (key, value) pairs, so
  // the reorganisation scatters one 8-byte word per key (measured 1.3 %
  // faster than two 4-byte scatters)
  static constexpr bool PACKED = PAIRS && KBITS == 32;

  static constexpr size_t al(size_t x) { return (x + 127) / 128 * 128; }
  // shared memory layout (bytes)
  static constexpr size_t stage_k = 0;                                      // tile keys + 16 B of span slack
  static constexpr size_t stage_v = al(stage_k + (size_t)T * sizeof(K) + 16);
  static constexpr size_t sorted = al(stage_v + (PAIRS ? (size_t)T * 4 + 16 : 0));
  static constexpr size_t sorted_bytes = al((size_t)T * (sizeof(K) + kVB));  // keys then values
  static constexpr size_t tables = sorted + 2 * sorted_bytes;              // [NR][256] lane masks, [NR][256] counts
  static constexpr size_t meta = tables + (size_t)NR * kRadix * 8;         // per sorted buffer: dstart[256], count[256]
  static constexpr size_t gbase = meta + 2 * 2 * kRadix * 4;               // writers: [256]
  static constexpr size_t scan = gbase + kRadix * 4;                       // rankers' scan scratch [32]
  static constexpr size_t ctx = scan + 32 * 4;                             // WsTile: staging, sorted 0, sorted 1
  static constexpr size_t bars = al(ctx + 3 * sizeof(WsTile));             // 7 mbarriers
  static constexpr size_t smem_bytes = bars + 7 * 8;
};

// Element j of a sorted buffer: key array then value array, or (key, value)
// pairs in PACKED mode.
template <typename C>
__device__ __forceinline__ void ws_put(typename C::K* sk, uint32_t* sv, uint32_t j, typename C::K k, uint32_t v) {
  if constexpr (C::PACKED) {
    reinterpret_cast<uint2*>(sk)[j] = make_uint2((uint32_t)k, v);
  } else {
    sk[j] = k;
    if (C::kVB) sv[j] = v;
  }
}
template <typename C>
__device__ __forceinline__ void ws_get(const typename C::K* sk, const uint32_t* sv, uint32_t j, typename C::K& k,
                                       uint32_t& v) {
  if constexpr (C::PACKED) {
    const uint2 kv = reinterpret_cast<const uint2*>(sk)[j];
    k = kv.x;
    v = kv.y;
  } else {
    k = sk[j];
    v = C::kVB ? sv[j] : 0u;
  }
}

constexpr int kBarRankers = 1;  // named barrier ids (0 is __syncthreads)
constexpr int kBarWriters = 2;
constexpr uint32_t kPipeWaitLimit = 1u << 22;

__device__ __forceinline__ void named_bar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// Named barrier that also returns whether any participating thread had p.
__device__ __forceinline__ bool named_bar_or(int id, int n, bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred a, b;\n\t"
      "setp.ne.u32 a, %1, 0;\n\t"
      "bar.red.or.pred b, %2, %3, a;\n\t"
      "selp.u32 %0, 1, 0, b;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)p), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Pipeline wait: phase `parity` of `bar`. Gives up (false) when the device
// status word is set (another role or block stopped) or after the poll limit
// (then it sets the timeout bit itself).
__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t parity, uint32_t* error) {
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 1023u) == 0u) {
      if (ld_relaxed_gpu(error) != 0u) return false;
      if (i >= kPipeWaitLimit) {
        atomicOr(error, kErrTimeout);
        return false;
      }
    }
  }
}

// Exclusive sum over the rankers' NRT threads (named barrier kBarRankers).
template <int NRT>
__device__ __forceinline__ uint32_t ranker_exclusive_sum(uint32_t v, uint32_t* tmp) {
  constexpr int NW = NRT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tmp[warp] = x;
  named_bar_sync(kBarRankers, NRT);
  if (warp == 0) {
    const uint32_t w = lane < NW ? tmp[lane] : 0u;
    uint32_t s = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < NW) tmp[lane] = s - w;
  }
  named_bar_sync(kBarRankers, NRT);
  return tmp[warp] + x - v;
}

// ------------------------------------------------------------------ staging

// Stages tile `tile` (none when past the end, or when the device status word
// is set) into the staging buffer and completes the staging mbarrier's next
// phase: with the bulk copies' bytes, or at once when the rankers will read
// the tile from global memory or there is no tile. Returns whether a tile was
// staged. Called by one ranker thread, when every ranker has read the
// previous tile out of the buffer.
template <int KBITS, bool PAIRS>
__device__ __forceinline__ bool ws_stage(const PassArgs& a, unsigned char* smem, uint32_t tile) {
  using C = WsConfig<KBITS, PAIRS>;
  using K = typename C::K;
  constexpr uint32_t T = C::T, kKeysPer16B = 16 / sizeof(K);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::bars);
  WsTile t{};
  t.tile = tile;
  const bool any = tile < a.num_tiles && ld_relaxed_gpu(a.error) == 0u;
  uint32_t kbytes = 0, vbytes = 0, ks = 0, vs = 0;
  if (any) {
    t.start = tile * T;
    t.count = min(T, a.n - t.start);
    if (a.use_bulk) {
      // the 16-byte-aligned span covering the tile, if it stays in the array
      ks = t.start & ~(kKeysPer16B - 1u);
      vs = t.start & ~3u;
      t.koff = t.start - ks;
      t.voff = t.start - vs;
      kbytes = ((t.koff + t.count) * (uint32_t)sizeof(K) + 15u) & ~15u;
      vbytes = ((t.voff + t.count) * 4u + 15u) & ~15u;
      t.bulk = (uint64_t)ks * sizeof(K) + kbytes <= (uint64_t)a.n * sizeof(K) &&
               (!PAIRS || (uint64_t)vs * 4u + vbytes <= (uint64_t)a.n * 4u);
    }
  }
  *reinterpret_cast<WsTile*>(smem + C::ctx) = t;
  if (t.bulk) {
    mbar_arrive_expect_tx(full, kbytes + (PAIRS ? vbytes : 0u));
    bulk_copy_g2s(smem + C::stage_k, static_cast<const K*>(a.keys_in) + ks, kbytes, full);
    if (PAIRS) bulk_copy_g2s(smem + C::stage_v, a.vals_in + vs, vbytes, full);
  } else {
    mbar_arrive(full);  // no copy: the rankers read the tile from global memory (or stop)
  }
  return any;
}

// Waits (bounded, whatever the status word says) for the staging phase
// `parity`, so that no bulk copy still writes into shared memory when the
// block exits.
__device__ __forceinline__ void ws_drain(uint64_t* full, uint32_t parity) {
  for (uint32_t i = 0; i < kPipeWaitLimit && !mbar_try_wait(full, parity); ++i) {
  }
}

// ------------------------------------------------------------------ rankers

template <int KBITS, bool PAIRS, int RANK, int FLIP, bool FULL>
__device__ __forceinline__ void ws_rank_tile(const PassArgs& a, unsigned char* smem, const WsTile& t, uint32_t b,
                                             uint32_t it, bool& stop, uint32_t& next, bool& more) {
  bool fail = false;  // this thread's wait for the sorted buffer gave up
  using C = WsConfig<KBITS, PAIRS>;
  using K = typename C::K;
  constexpr int NR = C::NR, IPT = C::IPT, NRT = C::NRT;
  const int rt = threadIdx.x, lane = rt & 31, warp = rt >> 5;
  const int shift = a.shift;
  const uint32_t mask = a.mask, dxor = a.digit_xor;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::bars);
  uint32_t* tables = reinterpret_cast<uint32_t*>(smem + C::tables);
  uint32_t* wmsk_all = tables;                  // [NR][256]
  uint32_t* wcnt_all = tables + NR * kRadix;    // [NR][256]
  uint32_t* meta = reinterpret_cast<uint32_t*>(smem + C::meta) + b * 2 * kRadix;
  uint32_t* dstart = meta;                      // [256]
  uint32_t* dcount = meta + kRadix;             // [256]
  uint32_t* scan = reinterpret_cast<uint32_t*>(smem + C::scan);
  K* sk = reinterpret_cast<K*>(smem + C::sorted + b * C::sorted_bytes);
  uint32_t* sv = reinterpret_cast<uint32_t*>(smem + C::sorted + b * C::sorted_bytes + (size_t)C::T * sizeof(K));
  const uint32_t count = t.count;
  const bool publish = (int64_t)t.tile != a.fault_tile;
  const bool head = t.tile == 0u;

  // 1. the tile into registers: warp-striped, batch i of warp w covers tile
  //    positions [w*IPT*32 + i*32, +32), so batch order and lane order are
  //    input order
  K key[IPT];
  uint32_t val[PAIRS ? IPT : 1];
  const uint32_t wbase = (uint32_t)warp * IPT * 32 + lane;
  K first;
  if (t.bulk) {
    const K* kt = reinterpret_cast<const K*>(smem + C::stage_k) + t.koff;
    const uint32_t* vt = reinterpret_cast<const uint32_t*>(smem + C::stage_v) + t.voff;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const uint32_t idx = wbase + i * 32;
      key[i] = load_transform<FLIP>((FULL || idx < count) ? kt[idx] : K(0));
      if (PAIRS) val[i] = (FULL || idx < count) ? vt[idx] : 0u;
    }
    first = load_transform<FLIP>(kt[0]);
  } else {
    const K* kg = static_cast<const K*>(a.keys_in) + t.start;
    const uint32_t* vg = PAIRS ? a.vals_in + t.start : nullptr;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const uint32_t idx = wbase + i * 32;
      key[i] = load_transform<FLIP>((FULL || idx < count) ? kg[idx] : K(0));
      if (PAIRS) val[i] = (FULL || idx < count) ? vg[idx] : 0u;
    }
    first = load_transform<FLIP>(kg[0]);
  }
  // homogeneous-tile test (Section 3, last paragraph of the kernel): any
  // digit bit differing from the first key's. The barrier also marks every
  // ranker's staged keys and values as read.
  const K digit_bits = (K)mask << shift;
  K differ = 0;
#pragma unroll
  for (int i = 0; i < IPT; ++i)
    if (FULL || wbase + i * 32 < count) differ |= (key[i] ^ first) & digit_bits;
  const bool homogeneous = !named_bar_or(kBarRankers, NRT, differ != 0);
  if (rt == 0) {
    // the staging buffer is free: stage the next tile, take the one after
    more = ws_stage<KBITS, PAIRS>(a, smem, next);
    if (more) next = atomicAdd(a.tile_counter, 1u);
  }

  // the next launch's status counters of this tile start at N
  if (a.status_clear && rt < kRadix)
    for (size_t row = t.tile; row < a.status_clear_rows; row += a.num_tiles) a.status_clear[row * kRadix + rt] = 0u;
  uint32_t* status = a.status + (size_t)t.tile * kRadix;
  const uint32_t d0 = digit_of(first, shift, mask, dxor);

  // the sorted buffer b is free once the writers finished tile it-2
  auto wait_buffer = [&]() {
    if (it >= 2 && !ws_wait(bars + 5 + b, ((it >> 1) - 1) & 1u, a.error)) fail = true;
  };

  if (homogeneous) {
    uint32_t c = 0;
    if (rt < kRadix) {
      c = (uint32_t)rt == d0 ? count : 0u;
      if (publish) st_relaxed_gpu(status + rt, ((head ? kFlagGlobal : kFlagLocal) << kStatusShift) | c);
    }
    wait_buffer();
    if (rt < kRadix) {
      dstart[rt] = 0u;
      dcount[rt] = c;
    }
    if (rt == 0) reinterpret_cast<WsTile*>(smem + C::ctx)[1 + b] = t;
    stop = named_bar_or(kBarRankers, NRT, fail);
    if (stop) return;
    if (rt == 0) mbar_arrive(bars + 1 + b);  // counts ready
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const uint32_t idx = wbase + i * 32;
      if (FULL || idx < count) ws_put<C>(sk, sv, idx, key[i], PAIRS ? val[i] : 0u);
    }
  } else {
    // 2. warp-level multi-split ranking (Section 3, WLMS); RANK is the
    //    ballot or the hybrid method here
    uint32_t* wmsk = wmsk_all + warp * kRadix;
    uint32_t* wc = wcnt_all + warp * kRadix;
    uint32_t rank2[IPT / 2 + 1];
    const uint32_t lane_bit = 1u << lane;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const bool valid = FULL || wbase + i * 32 < count;
      const bool smask = RANK == kRankHybrid && hybrid_uses_masks(i);
      const uint32_t r = wlms_rank<FULL>(wmsk, wc, digit_of(key[i], shift, mask, dxor), valid, lane_bit, smask);
      if (i & 1)
        rank2[i / 2] |= r << 16;
      else
        rank2[i / 2] = r;
    }
    named_bar_sync(kBarRankers, NRT);

    // 3. tile digit counts, published as (L, count) - or (G, count) by the
    //    first tile - before anything waits on the writers
    uint32_t c = 0;
    if (rt < kRadix) {
#pragma unroll
      for (int w = 0; w < NR; ++w) c += wcnt_all[w * kRadix + rt];
      if (publish) st_relaxed_gpu(status + rt, ((head ? kFlagGlobal : kFlagLocal) << kStatusShift) | c);
    }
    const uint32_t excl = ranker_exclusive_sum<NRT>(rt < kRadix ? c : 0u, scan);
    if (rt < kRadix) {
      uint32_t run = excl;
#pragma unroll
      for (int w = 0; w < NR; ++w) {
        const uint32_t cw = wcnt_all[w * kRadix + rt];
        wcnt_all[w * kRadix + rt] = run;
        run += cw;
      }
    }
    wait_buffer();
    if (rt < kRadix) {
      dstart[rt] = excl;
      dcount[rt] = c;
    }
    if (rt == 0) reinterpret_cast<WsTile*>(smem + C::ctx)[1 + b] = t;
    stop = named_bar_or(kBarRankers, NRT, fail);
    if (stop) return;
    // the counts are ready: the writers start this tile's look-back while
    // the keys are reorganised
    if (rt == 0) mbar_arrive(bars + 1 + b);

    // 4. local reorganisation into the sorted buffer: keys and values of
    //    each digit in input order, digits in ascending order
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const bool valid = FULL || wbase + i * 32 < count;
      if (valid) {
        const uint32_t r = (i & 1) ? (rank2[i / 2] >> 16) : (rank2[i / 2] & 0xFFFFu);
        const uint32_t p = wc[digit_of(key[i], shift, mask, dxor)] + r;
        if (p < C::T) ws_put<C>(sk, sv, p, key[i], PAIRS ? val[i] : 0u);
      }
    }
    // this warp's running counts start the next tile at zero
    __syncwarp();
#pragma unroll
    for (int j = 0; j < kRadix / 32; ++j) wc[j * 32 + lane] = 0u;
  }
  named_bar_sync(kBarRankers, NRT);
  if (rt == 0) {
    __threadfence_block();
    mbar_arrive(bars + 3 + b);  // keys and values reorganised: the writers copy them out
  }
}

template <int KBITS, bool PAIRS, int RANK, int FLIP>
__device__ void ws_rankers(const PassArgs& a, unsigned char* smem) {
  using C = WsConfig<KBITS, PAIRS>;
  constexpr int NRT = C::NRT;
  const int rt = threadIdx.x;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::bars);
  const WsTile* sctx = reinterpret_cast<const WsTile*>(smem + C::ctx);
  constexpr int R1 = RANK == kRankBallot ? kRankBallot : kRankHybrid;
  const bool ballots = RANK == kRankBallot || (RANK == kRankAdaptive && a.skew_flags && *a.skew_flags);

  // thread 0 stages the first tile and takes the id of the second
  uint32_t next = 0;
  bool more = false;
  if (rt == 0) {
    more = ws_stage<KBITS, PAIRS>(a, smem, atomicAdd(a.tile_counter, 1u));
    if (more) next = atomicAdd(a.tile_counter, 1u);
  }
  for (uint32_t it = 0;; ++it) {
    const uint32_t b = it & 1u;
    const bool staged = ws_wait(bars + 0, it & 1u, a.error);
    if (named_bar_or(kBarRankers, NRT, !staged)) {
      if (rt == 0) ws_drain(bars + 0, it & 1u);
      return;
    }
    const WsTile t = sctx[0];
    if (t.count == 0) {
      // end of the pass: hand the end marker to the writers through buffer b
      const bool fail = it >= 2 && !ws_wait(bars + 5 + b, ((it >> 1) - 1) & 1u, a.error);
      if (rt == 0) reinterpret_cast<WsTile*>(smem + C::ctx)[1 + b] = t;
      if (!named_bar_or(kBarRankers, NRT, fail) && rt == 0) mbar_arrive(bars + 1 + b);
      return;
    }
    // one uniform branch per tile between whole tile bodies: ballots only
    // (a skewed place, or the ballot variant) or the hybrid
    bool stop = false;
    if (t.count == (uint32_t)C::T) {
      if (ballots)
        ws_rank_tile<KBITS, PAIRS, kRankBallot, FLIP, true>(a, smem, t, b, it, stop, next, more);
      else
        ws_rank_tile<KBITS, PAIRS, R1, FLIP, true>(a, smem, t, b, it, stop, next, more);
    } else {
      if (ballots)
        ws_rank_tile<KBITS, PAIRS, kRankBallot, FLIP, false>(a, smem, t, b, it, stop, next, more);
      else
        ws_rank_tile<KBITS, PAIRS, R1, FLIP, false>(a, smem, t, b, it, stop, next, more);
    }
    if (stop) {
      // the tile staged for the next round may still be landing
      if (rt == 0) ws_drain(bars + 0, (it + 1) & 1u);
      return;
    }
  }
}

// ------------------------------------------------------------------ writers

// Decoupled look-back of digit d for tile t (Section 3, Figure 7): sums the
// preceding tiles' counters, up to kLookbackWindow per round trip, until a G
// counter or the first tile, then publishes (G, inclusive prefix). Returns
// the exclusive prefix. A wait past the poll limit records a timeout and
// still publishes, so the successors' walks end.
__device__ __forceinline__ uint32_t ws_walk(const PassArgs& a, uint32_t tile, int d, uint32_t own) {
  if (tile == 0u) return 0u;  // the first tile published (G, count) itself
  Lookback<kLookbackWindow> lb;
  lb.start(tile, 0u);
  lb.mine = (int64_t)tile != a.fault_tile ? a.status + (size_t)tile * kRadix + d : nullptr;
  lb.own = own;
  uint32_t spins = 0;
  while (!lb.done) {
    lb.issue(a.status, 0u, d);
    lb.consume();
    if (lb.done) break;
    if (++spins >= a.spin_limit) {
      atomicOr(a.error, kErrTimeout);
      break;
    }
    if ((spins & 255u) == 0 && (ld_relaxed_gpu(a.error) & kErrTimeout)) break;
  }
  if (!lb.done) lb.publish_global();
  return lb.exclusive;
}

template <int KBITS, bool PAIRS, int FLIP>
__device__ void ws_writers(const PassArgs& a, unsigned char* smem) {
  using C = WsConfig<KBITS, PAIRS>;
  using K = typename C::K;
  constexpr int NWT = C::NWT;
  const int wt = threadIdx.x - C::NRT;  // writer thread; threads 0..255 walk digit wt's chain
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::bars);
  uint32_t* gbase = reinterpret_cast<uint32_t*>(smem + C::gbase);
  const int shift = a.shift;
  const uint32_t mask = a.mask, dxor = a.digit_xor;
  const uint32_t bin_offset = wt < kRadix ? __ldg(a.bin_offsets + wt) : 0u;
  K* keys_out = static_cast<K*>(a.keys_out);
  uint32_t* vals_out = a.vals_out;
  const uint32_t out_len = a.out_total;

  for (uint32_t it = 0;; ++it) {
    const uint32_t b = it & 1u;
    // the tile's digit counts (the rankers are still reorganising it)
    const bool counted = ws_wait(bars + 1 + b, (it >> 1) & 1u, a.error);
    if (named_bar_or(kBarWriters, NWT, !counted)) break;
    const WsTile t = reinterpret_cast<const WsTile*>(smem + C::ctx)[1 + b];
    if (t.count == 0) break;
    const uint32_t* meta = reinterpret_cast<const uint32_t*>(smem + C::meta) + b * 2 * kRadix;
    if (wt < kRadix) {
      const uint32_t own = meta[kRadix + wt];
      const uint32_t exclusive = ws_walk(a, t.tile, wt, own);
      gbase[wt] = bin_offset + exclusive - meta[wt];
      if (a.carry_out && t.tile == a.num_tiles - 1) a.carry_out[wt] = bin_offset + exclusive + own;
    }
    // the reorganised keys and values
    const bool sorted = ws_wait(bars + 3 + b, (it >> 1) & 1u, a.error);
    if (named_bar_or(kBarWriters, NWT, !sorted)) break;

    // coalesced scatter of each bin run to its global bin
    const K* sk = reinterpret_cast<const K*>(smem + C::sorted + b * C::sorted_bytes);
    const uint32_t* sv =
        reinterpret_cast<const uint32_t*>(smem + C::sorted + b * C::sorted_bytes + (size_t)C::T * sizeof(K));
    if (t.count == (uint32_t)C::T) {
#pragma unroll 4
      for (int j = wt; j < C::T; j += NWT) {
        K k;
        uint32_t v;
        ws_get<C>(sk, sv, j, k, v);
        const uint32_t g = gbase[digit_of(k, shift, mask, dxor)] + j;
        if (g < out_len) {
          keys_out[g] = store_transform<FLIP>(k);
          if (PAIRS) vals_out[g] = v;
        }
      }
    } else {
      for (uint32_t j = wt; j < t.count; j += NWT) {
        K k;
        uint32_t v;
        ws_get<C>(sk, sv, j, k, v);
        const uint32_t g = gbase[digit_of(k, shift, mask, dxor)] + j;
        if (g < out_len) {
          keys_out[g] = store_transform<FLIP>(k);
          if (PAIRS) vals_out[g] = v;
        }
      }
    }
    named_bar_sync(kBarWriters, NWT);
    if (wt == 0) mbar_arrive(bars + 5 + b);  // buffer b free for the rankers' tile it+2
  }
}

// ------------------------------------------------------------------ kernel

template <int KBITS, bool PAIRS, int RANK, int FLIP>
__global__ void __launch_bounds__(WsConfig<KBITS, PAIRS>::NT, 1) binning_ws_kernel(PassArgs a) {
  using C = WsConfig<KBITS, PAIRS>;
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::bars);
  if (tid == 0) {
    mbar_init(bars + 0, 1);  // staging full: the staging thread's arrive (+ the copies' bytes)
    mbar_init(bars + 1, 1);  // buffer 0 / 1: the tile's digit counts ready (one ranker)
    mbar_init(bars + 2, 1);
    mbar_init(bars + 3, 1);  // buffer 0 / 1: keys and values reorganised (one ranker)
    mbar_init(bars + 4, 1);
    mbar_init(bars + 5, 1);  // buffer 0 / 1 free again (one writer)
    mbar_init(bars + 6, 1);
    fence_mbar_init();
  }
  // lane-mask and count tables start at zero (ranking leaves the masks at
  // zero; each warp zeroes its counts after its reorganisation)
  uint32_t* tables = reinterpret_cast<uint32_t*>(smem + C::tables);
  for (int i = tid; i < C::NR * kRadix * 2; i += C::NT) tables[i] = 0u;
  __syncthreads();
  if (warp < C::NR)
    ws_rankers<KBITS, PAIRS, RANK, FLIP>(a, smem);
  else
    ws_writers<KBITS, PAIRS, FLIP>(a, smem);
}

// Resident blocks of the persistent kernel: one per SM, at most one per tile.
int ws_grid(uint32_t num_tiles);

template <int KBITS, bool PAIRS, int RANK, int FLIP>
cudaError_t launch_binning_ws(const PassArgs& a, cudaStream_t s) {
  using C = WsConfig<KBITS, PAIRS>;
  cudaError_t e = cudaFuncSetAttribute(binning_ws_kernel<KBITS, PAIRS, RANK, FLIP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_bytes);
  if (e != cudaSuccess) return e;
  const int grid = ws_grid(a.num_tiles);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  binning_ws_kernel<KBITS, PAIRS, RANK, FLIP><<<grid, C::NT, C::smem_bytes, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ dispatch

template <int KBITS, bool PAIRS, int CFG, int RANK, int FLIP, bool SEG, int RB = kRadixBits>
cudaError_t launch_binning_one(const PassArgs& a, cudaStream_t s) {
  using C = BinningConfig<KBITS, PAIRS, CFG>;
  // set on every launch: an idempotent host-side attribute, so concurrent
  // callers on any device need no shared state
  cudaError_t e = cudaFuncSetAttribute(binning_kernel<KBITS, PAIRS, CFG, RANK, FLIP, SEG, RB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_bytes);
  if (e != cudaSuccess) return e;
  binning_kernel<KBITS, PAIRS, CFG, RANK, FLIP, SEG, RB><<<a.num_tiles, C::NT, C::smem_bytes, s>>>(a);
  return cudaGetLastError();
}

// Digits narrower than 8 bits (the digit-width sweep of Section 4, Table 2):
// tile geometry 0, adaptive ranking, one array; every payload and float
// transform mode. RB: bits per digit.
template <int KBITS, int RB>
cudaError_t launch_binning_rb_t(bool pairs, int flip, const PassArgs& a, cudaStream_t s) {
  switch ((pairs ? 4 : 0) | (flip & 3)) {
    case 0: return launch_binning_one<KBITS, false, 0, kRankAdaptive, 0, false, RB>(a, s);
    case 1: return launch_binning_one<KBITS, false, 0, kRankAdaptive, 1, false, RB>(a, s);
    case 2: return launch_binning_one<KBITS, false, 0, kRankAdaptive, 2, false, RB>(a, s);
    case 3: return launch_binning_one<KBITS, false, 0, kRankAdaptive, 3, false, RB>(a, s);
    case 4: return launch_binning_one<KBITS, true, 0, kRankAdaptive, 0, false, RB>(a, s);
    case 5: return launch_binning_one<KBITS, true, 0, kRankAdaptive, 1, false, RB>(a, s);
    case 6: return launch_binning_one<KBITS, true, 0, kRankAdaptive, 2, false, RB>(a, s);
    default: return launch_binning_one<KBITS, true, 0, kRankAdaptive, 3, false, RB>(a, s);
  }
}

template <int KBITS, bool PAIRS, int FLIP, int RANK, bool SEG>
cudaError_t launch_binning_flip_rank(const PassArgs& a, cudaStream_t s, int cfg) {
  switch (cfg) {
    case 1: return launch_binning_one<KBITS, PAIRS, 1, RANK, FLIP, SEG>(a, s);
    case 2: return launch_binning_one<KBITS, PAIRS, 2, RANK, FLIP, SEG>(a, s);
    case 3:
      // the persistent kernel serves one array (strips included); a batch
      // keeps geometry 0 (its plan is made with that tile)
      if (!SEG) return launch_binning_ws<KBITS, PAIRS, RANK, FLIP>(a, s);
      return launch_binning_one<KBITS, PAIRS, 0, RANK, FLIP, SEG>(a, s);
    default: return launch_binning_one<KBITS, PAIRS, 0, RANK, FLIP, SEG>(a, s);
  }
}

// All tile geometries (0-2: one block per tile; 3: the persistent
// warp-specialised kernel) and the ranking variants for one (width, payload,
// float transform mode, single array / segmented). The grid is a.num_tiles
// blocks (an upper bound in segmented mode; blocks beyond the last tile exit).
template <int KBITS, bool PAIRS, int FLIP, bool SEG>
cudaError_t launch_binning_flip(const PassArgs& a, cudaStream_t s, int cfg, int rank) {
  switch (rank) {
    case kRankAdaptive: return launch_binning_flip_rank<KBITS, PAIRS, FLIP, kRankAdaptive, SEG>(a, s, cfg);
    case kRankHybrid: return launch_binning_flip_rank<KBITS, PAIRS, FLIP, kRankHybrid, SEG>(a, s, cfg);
    default: return launch_binning_flip_rank<KBITS, PAIRS, FLIP, kRankBallot, SEG>(a, s, cfg);
  }
}

template <int KBITS, bool PAIRS>
uint32_t tile_keys_t(int cfg) {
  switch (cfg) {
    case 1: return BinningConfig<KBITS, PAIRS, 1>::T;
    case 2: return BinningConfig<KBITS, PAIRS, 2>::T;
    case 3: return WsConfig<KBITS, PAIRS>::T;
    default: return BinningConfig<KBITS, PAIRS, 0>::T;
  }
}

}  // namespace onesweep
