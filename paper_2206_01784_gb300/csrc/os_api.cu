// Host driver and C ABI of the GB300 Onesweep sort (arXiv 2206.01784).
//
// Section 3, "High-level description": the sort is three phases, each a GPU
// kernel - one histogram pass over all digit places, an exclusive sum of each
// histogram, then p chained-scan digit-binning passes. Here phases 1 and 2
// share one launch; the driver validates arguments, carves the caller's
// workspace, zeroes its small header with one memset and enqueues the
// launches on the caller's stream. Nothing is allocated and nothing waits on
// the host.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "../../include/onesweep.h"
#include "../../include/onesweep_debug.h"
#include "os_common.cuh"
#include "os_internal.h"

namespace onesweep {

#define OS_DECLARE_BINNING_MODE(KB, PR, M)                                                  \
  cudaError_t launch_binning##KB##_##PR##_f0_##M(int, int, const PassArgs&, cudaStream_t);   \
  cudaError_t launch_binning##KB##_##PR##_f1_##M(int, int, const PassArgs&, cudaStream_t);   \
  cudaError_t launch_binning##KB##_##PR##_f2_##M(int, int, const PassArgs&, cudaStream_t);   \
  cudaError_t launch_binning##KB##_##PR##_f3_##M(int, int, const PassArgs&, cudaStream_t);
#define OS_DECLARE_BINNING(KB, PR)           \
  OS_DECLARE_BINNING_MODE(KB, PR, single)    \
  OS_DECLARE_BINNING_MODE(KB, PR, seg)       \
  uint32_t binning_tile_keys##KB##_##PR(int cfg);
OS_DECLARE_BINNING(32, pairs)
OS_DECLARE_BINNING(32, keys)
OS_DECLARE_BINNING(64, pairs)
OS_DECLARE_BINNING(64, keys)
#undef OS_DECLARE_BINNING
#undef OS_DECLARE_BINNING_MODE

using BinningLaunch = cudaError_t (*)(int, int, const PassArgs&, cudaStream_t);

#define OS_BINNING_ROW(KB, PR, M) \
  {launch_binning##KB##_##PR##_f0_##M, launch_binning##KB##_##PR##_f1_##M, launch_binning##KB##_##PR##_f2_##M, \
   launch_binning##KB##_##PR##_f3_##M}
// [segmented][64-bit][pairs][float transform mode]
const BinningLaunch kBinningLaunch[2][2][2][4] = {
    {{OS_BINNING_ROW(32, keys, single), OS_BINNING_ROW(32, pairs, single)},
     {OS_BINNING_ROW(64, keys, single), OS_BINNING_ROW(64, pairs, single)}},
    {{OS_BINNING_ROW(32, keys, seg), OS_BINNING_ROW(32, pairs, seg)},
     {OS_BINNING_ROW(64, keys, seg), OS_BINNING_ROW(64, pairs, seg)}}};
#undef OS_BINNING_ROW

// Digits narrower than 8 bits (os_sort_options.radix_bits 5-7)
#define OS_DECLARE_RB(RB)                                                                 \
  cudaError_t launch_binning_rb##RB##_32(bool, int, const PassArgs&, cudaStream_t);       \
  cudaError_t launch_binning_rb##RB##_64(bool, int, const PassArgs&, cudaStream_t);
OS_DECLARE_RB(5)
OS_DECLARE_RB(6)
OS_DECLARE_RB(7)
#undef OS_DECLARE_RB
using BinningLaunchRb = cudaError_t (*)(bool, int, const PassArgs&, cudaStream_t);
constexpr int kMinRadixBits = 5;
// [64-bit][radix bits - kMinRadixBits]
const BinningLaunchRb kBinningLaunchRb[2][3] = {
    {launch_binning_rb5_32, launch_binning_rb6_32, launch_binning_rb7_32},
    {launch_binning_rb5_64, launch_binning_rb6_64, launch_binning_rb7_64}};
constexpr int kMaxPlaces = 16;  // 64-bit keys in 5-bit digits: 13 places

// Binning kernel variants: tile geometry (4) x digit-ranking method (3);
// variant v uses geometry v % 4 and ranking v / 4 (0: one ballot per digit
// bit; 1: adaptive - ballots where the place is skewed, else the hybrid;
// 2: hybrid - shared-memory lane masks on two of every three batches, ballots
// on the third).
// Geometries 0-2 run one block per tile; geometry 3 is the persistent,
// warp-specialised kernel (os_binning_ws.cuh), for single arrays only.
constexpr int kGeometries = 4;
constexpr int kPersistentGeometry = 3;
constexpr int kTileConfigs = 3 * kGeometries;

// Active variant per (key width, keys only / pairs, size bucket); set by
// os_set_tile_config / os_set_tile_config_bucket (the autotuner's hooks) and
// read once per sort when it is planned, with atomic loads and stores (a
// sort may also name its variant itself: os_sort_*_ex).
// Defaults: geometry 0 with adaptive ranking (the fastest measured on GB300
// for 32-bit keys at 2^28 across the key distributions), and for 64-bit keys
// of the largest bucket the persistent warp-specialised geometry with
// adaptive ranking (64-bit pairs at 2^27: 0.926 against 0.970 ms per pass;
// 2^24: 0.125 against 0.132; keys only 0.824 against 0.840; 3 % slower on
// q = 3 keys).
constexpr int kDefaultTileConfig = kGeometries + 0;
constexpr int kDefault64LargeConfig = kGeometries + kPersistentGeometry;
constexpr int kSizeBuckets = 4;  // n < 2^16, < 2^20, < 2^24, larger
#define OS_FOUR_DEFAULTS {kDefaultTileConfig, kDefaultTileConfig, kDefaultTileConfig, kDefaultTileConfig}
#define OS_FOUR_DEFAULTS_64 {kDefaultTileConfig, kDefaultTileConfig, kDefaultTileConfig, kDefault64LargeConfig}
int g_tile_cfg[2][2][kSizeBuckets] = {{OS_FOUR_DEFAULTS, OS_FOUR_DEFAULTS}, {OS_FOUR_DEFAULTS_64, OS_FOUR_DEFAULTS_64}};
#undef OS_FOUR_DEFAULTS
#undef OS_FOUR_DEFAULTS_64

int size_bucket(uint64_t n) { return n < (1u << 16) ? 0 : n < (1u << 20) ? 1 : n < (1u << 24) ? 2 : 3; }

// Process-wide digit width per (key width, payload, size bucket), for sorts
// whose options leave radix_bits at 0 (the autotuner sets it).
std::atomic<int> g_radix_bits[2][2][kSizeBuckets];
int get_radix_bits(int key_bits, bool pairs, int bucket) {
  const int v = g_radix_bits[key_bits == 64][pairs][bucket].load(std::memory_order_relaxed);
  return v == 0 ? kRadixBits : v;
}

int get_tile_cfg(int key_bits, bool pairs, int bucket) {
  return __atomic_load_n(&g_tile_cfg[key_bits == 64][pairs][bucket], __ATOMIC_RELAXED);
}
void set_tile_cfg(int key_bits, bool pairs, int bucket, int cfg) {
  __atomic_store_n(&g_tile_cfg[key_bits == 64][pairs][bucket], cfg, __ATOMIC_RELAXED);
}

uint32_t tile_keys_for(int key_bits, bool pairs, int cfg) {
  const int geo = cfg % kGeometries;
  if (key_bits == 32) return pairs ? binning_tile_keys32_pairs(geo) : binning_tile_keys32_keys(geo);
  return pairs ? binning_tile_keys64_pairs(geo) : binning_tile_keys64_keys(geo);
}

int binning_config(int key_bits, bool pairs, int bucket) { return get_tile_cfg(key_bits, pairs, bucket); }

// Smallest tile over all geometries: workspaces are sized for it, so any
// geometry fits a workspace sized once.
uint32_t min_tile_keys(int key_bits, bool pairs) {
  uint32_t t = tile_keys_for(key_bits, pairs, 0);
  for (int c = 1; c < kGeometries; ++c) {
    const uint32_t u = tile_keys_for(key_bits, pairs, c);
    if (u < t) t = u;
  }
  return t;
}

cudaError_t launch_binning(int key_bits, bool pairs, int cfg, const PassArgs& a, cudaStream_t s, int radix_bits) {
  const int flip = (a.flip_in ? 1 : 0) | (a.flip_out ? 2 : 0);
  const int seg = a.seg_offsets != nullptr;
  if (radix_bits != kRadixBits) {
    if (seg || radix_bits < kMinRadixBits || radix_bits > kRadixBits) return cudaErrorInvalidValue;
    return kBinningLaunchRb[key_bits == 64][radix_bits - kMinRadixBits](pairs, flip, a, s);
  }
  return kBinningLaunch[seg][key_bits == 64][pairs][flip](cfg % kGeometries, cfg / kGeometries, a, s);
}

namespace {

// Section 3, "Handling very large problems": the chained scan keeps 30-bit
// counts, so a pass over more than kStripKeys keys runs strip by strip (one
// launch each, every strip its own look-back chain); 32-bit output indices
// then bound n below 2^32.
constexpr uint64_t kMaxKeys = 1ull << 32;
constexpr uint64_t kStripKeys = (1ull << 30) - 1;  // every count of a strip fits 30 bits
constexpr uint64_t kMinStripKeys = 1ull << 16;
std::atomic<uint64_t> g_strip_keys{kStripKeys};  // shorter strips: os_debug_set_strip_keys
constexpr size_t kAlign = 256;
constexpr uint32_t kDefaultSpinLimit = 1u << 22;

// Header layout: word 0 device status, word 1 done counter of the histogram
// kernel, words 16..23 tile counters of a batch sort's binning passes (a
// single-array sort keeps one counter per launch after the histograms).
constexpr size_t kHeaderBytes = 256;
constexpr size_t kDoneWord = 1;
constexpr size_t kTileCounterWord = 16;
constexpr size_t kSkewWord = 32;  // 16 skewed-place flags of a single sort

// Test hooks (onesweep_debug.h), read once per sort when it is planned.
std::atomic<int64_t> g_fault_tile{-1};
std::atomic<uint32_t> g_spin_limit{kDefaultSpinLimit};

// Launch timing (os_profile_start / os_profile_stop): a table guarded by a
// lock; g_prof_on lets sorts skip the lock while timing is off.
struct ProfiledLaunch {
  cudaEvent_t start, stop;
  int kernel, pass;
};
std::mutex g_prof_mutex;
std::atomic<bool> g_prof_on{false};
ProfiledLaunch* g_prof = nullptr;
int g_prof_capacity = 0;
int g_prof_used = 0;
int g_prof_seen = 0;

// Records the start event of a launch if profiling is on; returns its slot.
int prof_begin(int kernel, int pass, cudaStream_t s) {
  if (!g_prof_on.load(std::memory_order_acquire)) return -1;
  std::lock_guard<std::mutex> lock(g_prof_mutex);
  if (!g_prof) return -1;
  ++g_prof_seen;
  if (g_prof_used >= g_prof_capacity) return -1;
  ProfiledLaunch& p = g_prof[g_prof_used];
  p.kernel = kernel;
  p.pass = pass;
  if (cudaEventRecord(p.start, s) != cudaSuccess) return -1;
  return g_prof_used++;
}

void prof_end(int slot, cudaStream_t s) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lock(g_prof_mutex);
  if (g_prof && slot < g_prof_capacity) cudaEventRecord(g_prof[slot].stop, s);
}

size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// key_type is a key type, optionally with OS_SORT_DESCENDING OR'd in.
bool known_flags(int key_type) { return (key_type & ~0xFF & ~OS_SORT_DESCENDING) == 0; }
bool is_descending(int key_type) { return (key_type & OS_SORT_DESCENDING) != 0; }

int key_bits_of(int key_type) {
  if (!known_flags(key_type)) return 0;
  switch (key_type & 0xFF) {
    case OS_KEY_U32:
    case OS_KEY_F32:
    case OS_KEY_I32: return 32;
    case OS_KEY_U64:
    case OS_KEY_F64:
    case OS_KEY_I64: return 64;
    default: return 0;
  }
}

bool is_float(int key_type) { return (key_type & 0xFF) == OS_KEY_F32 || (key_type & 0xFF) == OS_KEY_F64; }

// Signed keys sort as their bits with the sign bit inverted (two's complement
// order). Only the most significant place holds the sign bit, so instead of
// transforming keys, that place's digit gets its high bit inverted - when the
// sorted range reaches the sign bit.
uint32_t signed_top_xor(int key_type, int begin_bit, int end_bit, int radix_bits = kRadixBits) {
  const int kb = key_bits_of(key_type);
  const int base = key_type & 0xFF;
  if ((base != OS_KEY_I32 && base != OS_KEY_I64) || end_bit != kb || end_bit <= begin_bit) return 0u;
  const int places = (end_bit - begin_bit + radix_bits - 1) / radix_bits;
  const int top_width = end_bit - (begin_bit + radix_bits * (places - 1));
  return 1u << (top_width - 1);
}

struct Plan {
  int key_bits = 0;
  bool pairs = false;
  int bucket = 0;
  int cfg = 0;               // binning variant (geometry + ranking)
  int radix_bits = kRadixBits;  // d: bits per digit place
  int places = 0;
  int64_t fault_tile = -1;   // test hooks, read once
  uint32_t spin_limit = 0;
  uint32_t tile = 0;
  uint32_t tiles = 0;        // tiles of a whole pass
  uint64_t strip = 0;        // keys per strip (a multiple of the tile)
  uint32_t strips = 0;       // strips per pass
  size_t counters = 0;       // tile counters, one per launch
  size_t carry = 0;          // two [256] arrays of strip bin bases
  os_workspace_layout layout{};
};

// cfg_override: the caller's binning variant, or -1 for the process-wide one.
// radix_bits: bits per digit place (5-8; narrower digits use tile variant 4,
// geometry 0 with adaptive ranking), or 0 for the process-wide one (8 when
// the caller names another variant).
int make_plan(int key_type, uint64_t n, int value_bytes, int begin_bit, int end_bit, Plan* plan,
              int cfg_override = -1, int radix_bits = 0) {
  const int kb = key_bits_of(key_type);
  if (kb == 0) return OS_ERR_INVALID_ARG;
  if (value_bytes != 0 && value_bytes != 4) return OS_ERR_INVALID_ARG;
  if (begin_bit < 0 || end_bit > kb || begin_bit > end_bit) return OS_ERR_INVALID_ARG;
  if (n >= kMaxKeys) return OS_ERR_TOO_LARGE;
  plan->key_bits = kb;
  plan->pairs = value_bytes == 4;
  if (radix_bits == 0) {
    radix_bits = get_radix_bits(kb, plan->pairs, size_bucket(n));
    if (cfg_override >= 0 && cfg_override != kGeometries) radix_bits = kRadixBits;
  }
  if (radix_bits < kMinRadixBits || radix_bits > kRadixBits) return OS_ERR_INVALID_ARG;
  plan->radix_bits = radix_bits;
  plan->places = (end_bit - begin_bit + radix_bits - 1) / radix_bits;
  plan->bucket = size_bucket(n);
  // the variant is read once: every launch of this sort uses the same one
  if (cfg_override >= kTileConfigs) return OS_ERR_INVALID_ARG;
  plan->cfg = cfg_override >= 0 ? cfg_override : binning_config(kb, plan->pairs, plan->bucket);
  if (radix_bits != kRadixBits) {
    if (cfg_override >= 0 && cfg_override != kGeometries) return OS_ERR_INVALID_ARG;
    plan->cfg = kGeometries;  // geometry 0, adaptive ranking
  }
  plan->fault_tile = g_fault_tile.load(std::memory_order_relaxed);
  plan->spin_limit = g_spin_limit.load(std::memory_order_relaxed);
  plan->tile = tile_keys_for(kb, plan->pairs, plan->cfg);
  plan->tiles = (uint32_t)((n + plan->tile - 1) / plan->tile);
  // strips of equal length (whole tiles, at most the strip limit), so that no
  // launch is much shorter than the next one, whose status rows it clears
  const uint64_t max_strip = g_strip_keys.load(std::memory_order_relaxed) / plan->tile * plan->tile;
  const uint64_t want = n == 0 ? 1u : (n + max_strip - 1) / max_strip;
  uint64_t strip = (n + want - 1) / want;
  strip = (strip + plan->tile - 1) / plan->tile * plan->tile;
  plan->strip = strip;
  plan->strips = n == 0 ? 1u : (uint32_t)((n + strip - 1) / strip);
  // status slabs: rows for the largest launch (at most one strip of the
  // smallest tile of any geometry, so every geometry fits)
  const uint32_t min_tile = min_tile_keys(kb, plan->pairs);
  const uint64_t launch_keys = n < kStripKeys ? n : kStripKeys;
  const uint64_t max_tiles = (launch_keys + min_tile - 1) / min_tile;
  // one tile counter per launch: kMaxPlaces places x strips, for any strip length the
  // test hook allows (>= kMinStripKeys rounded down to a tile of < 2^15 keys,
  // then balanced: longer than n / (n / 2^15 + 1) keys; a workspace sized
  // once always fits)
  const uint64_t max_strips = n / (kMinStripKeys / 2) + 2;
  os_workspace_layout& L = plan->layout;
  std::memset(&L, 0, sizeof(L));
  size_t off = kHeaderBytes;
  L.histogram_offset = off;
  off = round_up(off + (size_t)kMaxPlaces * kRadix * 4);
  plan->counters = off;
  off = round_up(off + (size_t)kMaxPlaces * max_strips * 4);
  L.bin_offset_offset = off;
  off = round_up(off + (size_t)kMaxPlaces * kRadix * 4);
  plan->carry = off;
  off = round_up(off + (size_t)2 * kRadix * 4);
  const size_t slab = (size_t)max_tiles * kRadix * 4;
  L.status_offset[0] = off;
  off = round_up(off + slab);
  L.status_offset[1] = off;
  off = round_up(off + (plan->places > 1 ? slab : 0));
  L.alt_keys_offset = off;
  off = round_up(off + (plan->places > 1 ? (size_t)n * (kb / 8) : 0));
  L.alt_values_offset = off;
  off = round_up(off + (plan->places > 1 && plan->pairs ? (size_t)n * 4 : 0));
  L.total_bytes = off;
  L.tile_keys = plan->tile;
  L.num_tiles = plan->tiles;
  L.num_places = (uint32_t)plan->places;
  return OS_OK;
}

bool overlaps(const void* a, size_t abytes, const void* b, size_t bbytes) {
  if (!a || !b || abytes == 0 || bbytes == 0) return false;
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + bbytes && y < x + abytes;
}

}  // namespace

// SM count of the current device, cached per device (one atomic word each, so
// concurrent callers on different devices never mix their values).
int device_sm_count() {
  constexpr int kMaxCachedDevices = 64;
  static std::atomic<int> cache[kMaxCachedDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (dev >= 0 && dev < kMaxCachedDevices) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (dev >= 0 && dev < kMaxCachedDevices) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

int ws_grid(uint32_t num_tiles) {
  const int sms = device_sm_count();
  if (sms <= 0) return 0;
  return num_tiles < (uint32_t)sms ? (int)num_tiles : sms;
}

namespace {

// Phases 1 + 2 into the workspace (header already zeroed).
int run_histogram(const Plan& plan, int key_type, const void* keys, uint64_t n, int begin_bit, int end_bit,
                  char* ws, bool clear_slab0, cudaStream_t s) {
  HistArgs h{};
  h.keys = keys;
  h.n = n;
  h.flip = is_float(key_type);
  h.num_places = plan.places;
  h.radix_bits = plan.radix_bits;
  h.begin_bit = begin_bit;
  h.end_bit = end_bit;
  h.hist = reinterpret_cast<uint32_t*>(ws + plan.layout.histogram_offset);
  h.offsets = reinterpret_cast<uint32_t*>(ws + plan.layout.bin_offset_offset);
  h.done_counter = reinterpret_cast<uint32_t*>(ws) + kDoneWord;
  h.clear = clear_slab0 ? reinterpret_cast<uint32_t*>(ws + plan.layout.status_offset[0]) : nullptr;
  // the first launch's rows (the first strip's tiles)
  const uint64_t first_tiles = (plan.strip < n ? plan.strip : n + plan.tile - 1) / plan.tile;
  h.clear_words = clear_slab0 ? first_tiles * kRadix : 0;
  h.skew = reinterpret_cast<uint32_t*>(ws) + kSkewWord;
  h.top_xor = signed_top_xor(key_type, begin_bit, end_bit, plan.radix_bits);
  h.descending = is_descending(key_type) ? 1u : 0u;
  const int sms = device_sm_count();
  if (sms <= 0) return OS_ERR_CUDA;
  const int slot = prof_begin(0, -1, s);
  const cudaError_t e = launch_histogram(plan.key_bits, h, sms, s);
  prof_end(slot, s);
  return e == cudaSuccess ? OS_OK : OS_ERR_CUDA;
}

int run_sort(int key_type, const void* keys_in, void* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
             uint64_t n, int begin_bit, int end_bit, void* ws, size_t ws_bytes, void* stream, int cfg_override = -1,
             int radix_bits = 0) {
  const bool pairs = vals_in != nullptr || vals_out != nullptr;
  if (pairs && (vals_in == nullptr || vals_out == nullptr)) return OS_ERR_INVALID_ARG;
  Plan plan;
  int rc = make_plan(key_type, n, pairs ? 4 : 0, begin_bit, end_bit, &plan, cfg_override, radix_bits);
  if (rc != OS_OK) return rc;
  if (n == 0) return OS_OK;
  const size_t kbytes = (size_t)n * (plan.key_bits / 8);
  const size_t vbytes = pairs ? (size_t)n * 4 : 0;
  if (!keys_in || !keys_out) return OS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(keys_in) % (plan.key_bits / 8) ||
      reinterpret_cast<uintptr_t>(keys_out) % (plan.key_bits / 8))
    return OS_ERR_INVALID_ARG;
  if (pairs && (reinterpret_cast<uintptr_t>(vals_in) % 4 || reinterpret_cast<uintptr_t>(vals_out) % 4))
    return OS_ERR_INVALID_ARG;
  if (!ws || ws_bytes < plan.layout.total_bytes) return OS_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % 16) return OS_ERR_INVALID_ARG;
  if (overlaps(keys_in, kbytes, keys_out, kbytes) || overlaps(keys_in, kbytes, ws, plan.layout.total_bytes) ||
      overlaps(keys_out, kbytes, ws, plan.layout.total_bytes))
    return OS_ERR_INVALID_ARG;
  if (pairs) {
    const void* bufs[4] = {keys_in, keys_out, vals_in, vals_out};
    const size_t sizes[4] = {kbytes, kbytes, vbytes, vbytes};
    for (int i = 0; i < 4; ++i)
      for (int j = i + 1; j < 4; ++j)
        if (overlaps(bufs[i], sizes[i], bufs[j], sizes[j])) return OS_ERR_INVALID_ARG;
    if (overlaps(vals_in, vbytes, ws, plan.layout.total_bytes) ||
        overlaps(vals_out, vbytes, ws, plan.layout.total_bytes))
      return OS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);

  if (plan.places == 0) {  // empty bit range: a plain copy
    if (cudaMemsetAsync(w, 0, 4, s) != cudaSuccess) return OS_ERR_CUDA;
    if (cudaMemcpyAsync(keys_out, keys_in, kbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return OS_ERR_CUDA;
    if (pairs && cudaMemcpyAsync(vals_out, vals_in, vbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return OS_ERR_CUDA;
    return OS_OK;
  }

  // zero: status word, done counter, histograms, this sort's tile counters
  const size_t zero_bytes = plan.counters + (size_t)plan.places * plan.strips * 4;
  if (cudaMemsetAsync(w, 0, zero_bytes, s) != cudaSuccess) return OS_ERR_CUDA;
  rc = run_histogram(plan, key_type, keys_in, n, begin_bit, end_bit, w, true, s);
  if (rc != OS_OK) return rc;

  uint32_t* header = reinterpret_cast<uint32_t*>(w);
  const uint32_t* offsets = reinterpret_cast<const uint32_t*>(w + plan.layout.bin_offset_offset);
  void* alt_keys = w + plan.layout.alt_keys_offset;
  uint32_t* alt_vals = reinterpret_cast<uint32_t*>(w + plan.layout.alt_values_offset);
  const bool aligned_in = reinterpret_cast<uintptr_t>(keys_in) % 16 == 0 &&
                          (!pairs || reinterpret_cast<uintptr_t>(vals_in) % 16 == 0);
  const bool aligned_out = reinterpret_cast<uintptr_t>(keys_out) % 16 == 0 &&
                           (!pairs || reinterpret_cast<uintptr_t>(vals_out) % 16 == 0);

  const size_t kbytes_per_key = plan.key_bits / 8;
  uint32_t* counters = reinterpret_cast<uint32_t*>(w + plan.counters);
  uint32_t* carry = reinterpret_cast<uint32_t*>(w + plan.carry);  // two [256] arrays
  auto strip_len = [&](uint32_t st) {
    const uint64_t lo = (uint64_t)st * plan.strip;
    return (uint32_t)((n - lo) < plan.strip ? (n - lo) : plan.strip);
  };
  auto strip_tiles = [&](uint32_t st) { return (strip_len(st) + plan.tile - 1) / plan.tile; };
  const uint32_t launches = (uint32_t)plan.places * plan.strips;

  const void* src_k = keys_in;
  const uint32_t* src_v = vals_in;
  bool src_aligned = aligned_in;
  uint32_t launch = 0;
  for (int pass = 0; pass < plan.places; ++pass) {
    // ping-pong so that the last pass writes keys_out
    const bool to_out = ((plan.places - 1 - pass) % 2) == 0;
    void* dst_k = to_out ? keys_out : alt_keys;
    uint32_t* dst_v = to_out ? vals_out : alt_vals;
    for (uint32_t st = 0; st < plan.strips; ++st, ++launch) {
      const uint64_t lo = (uint64_t)st * plan.strip;
      PassArgs a{};
      a.keys_in = static_cast<const char*>(src_k) + lo * kbytes_per_key;
      a.keys_out = dst_k;
      a.vals_in = pairs ? src_v + lo : nullptr;
      a.vals_out = pairs ? dst_v : nullptr;
      a.n = strip_len(st);
      a.out_total = (uint32_t)n;
      a.num_tiles = strip_tiles(st);
      a.shift = begin_bit + plan.radix_bits * pass;
      const int width = end_bit - a.shift < plan.radix_bits ? end_bit - a.shift : plan.radix_bits;
      a.mask = (1u << width) - 1u;
      a.flip_in = is_float(key_type) && pass == 0;
      a.flip_out = is_float(key_type) && pass == plan.places - 1;
      a.use_bulk = src_aligned ? 1 : 0;
      // strip 0 starts at the global bin offsets; strip st at the bases strip
      // st-1 left in carry[(st-1) & 1]
      a.bin_offsets = st == 0 ? offsets + pass * kRadix : carry + ((st - 1) & 1) * kRadix;
      a.carry_out = st + 1 < plan.strips ? carry + (st & 1) * kRadix : nullptr;
      a.status = reinterpret_cast<uint32_t*>(w + plan.layout.status_offset[launch & 1]);
      a.status_clear = launch + 1 < launches
                           ? reinterpret_cast<uint32_t*>(w + plan.layout.status_offset[(launch + 1) & 1])
                           : nullptr;
      a.status_clear_rows = launch + 1 < launches ? strip_tiles((st + 1) % plan.strips) : 0u;
      if (a.status_clear_rows < a.num_tiles) a.status_clear_rows = a.num_tiles;
      a.tile_counter = counters + launch;
      a.error = header;
      a.spin_limit = plan.spin_limit;
      a.fault_tile = plan.fault_tile;
      a.skew_flags = header + kSkewWord + pass;
      // signed keys: the top place's high digit bit inverted; descending:
      // every digit complemented within its place
      a.digit_xor = (pass == plan.places - 1 ? signed_top_xor(key_type, begin_bit, end_bit, plan.radix_bits) : 0u) ^
                    (is_descending(key_type) ? a.mask : 0u);
      if (pass >= kMaxPlaces) {
        // more places cannot happen with >= 5-bit digits of <= 64-bit keys
        return OS_ERR_INVALID_ARG;
      }
      const int slot = prof_begin(1, pass, s);
      const cudaError_t e = launch_binning(plan.key_bits, pairs, plan.cfg, a, s, plan.radix_bits);
      prof_end(slot, s);
      if (e != cudaSuccess) return OS_ERR_CUDA;
    }
    src_k = dst_k;
    src_v = dst_v;
    src_aligned = to_out ? aligned_out : true;
  }
  return OS_OK;
}

// ---------------------------------------------------------------- batches

constexpr uint32_t kHistChunk = 32768;         // keys per histogram work item of a batch
constexpr uint64_t kMaxBatchKeys = 1ull << 31;  // total keys of a batch (32-bit indices)
constexpr uint64_t kMaxSegments = 1ull << 24;

// Batch header words (same header as a single sort): 0 status, 2 binning
// tiles, 3 histogram items, 4 invalid-offsets flag, 16.. tile counters.
constexpr size_t kTotalsWord = 2;

struct BatchPlan {
  int key_bits = 0;
  bool pairs = false;
  int bucket = 0;
  int cfg = 0;  // binning variant
  int64_t fault_tile = -1;  // test hooks, read once
  uint32_t spin_limit = 0;
  int places = 0;
  uint32_t tile = 0, small_max = 0;
  uint64_t max_tiles = 0, max_items = 0;
  size_t seg_done = 0, seg_skew = 0, seg_hist = 0, zero_end = 0, seg_bin_offsets = 0, tile_base = 0, hist_base = 0;
  size_t tile_seg = 0, hist_seg = 0, status[2] = {0, 0}, alt_keys = 0, alt_vals = 0, total = 0;
};

int make_batch_plan(int key_type, uint64_t n_total, int64_t num_segments, int value_bytes, int begin_bit,
                    int end_bit, BatchPlan* bp, int cfg_override = -1) {
  const int kb = key_bits_of(key_type);
  if (kb == 0 || num_segments < 0) return OS_ERR_INVALID_ARG;
  if (value_bytes != 0 && value_bytes != 4) return OS_ERR_INVALID_ARG;
  if (begin_bit < 0 || end_bit > kb || begin_bit > end_bit) return OS_ERR_INVALID_ARG;
  if (n_total >= kMaxBatchKeys || (uint64_t)num_segments > kMaxSegments) return OS_ERR_TOO_LARGE;
  const uint64_t S = (uint64_t)num_segments;
  bp->key_bits = kb;
  bp->pairs = value_bytes == 4;
  bp->places = (end_bit - begin_bit + kRadixBits - 1) / kRadixBits;
  bp->bucket = size_bucket(S > 0 ? n_total / S : n_total);  // by the mean segment length
  if (cfg_override >= kTileConfigs) return OS_ERR_INVALID_ARG;
  bp->cfg = cfg_override >= 0 ? cfg_override : binning_config(kb, bp->pairs, bp->bucket);
  bp->fault_tile = g_fault_tile.load(std::memory_order_relaxed);
  bp->spin_limit = g_spin_limit.load(std::memory_order_relaxed);
  // the persistent kernel serves single arrays: a batch runs geometry 0 with
  // the same ranking
  if (bp->cfg % kGeometries == kPersistentGeometry) bp->cfg -= kPersistentGeometry;
  bp->tile = tile_keys_for(kb, bp->pairs, bp->cfg);
  bp->small_max = batch_local_capacity(kb, bp->pairs);
  const uint32_t min_tile = min_tile_keys(kb, bp->pairs);
  bp->max_tiles = (n_total + min_tile - 1) / min_tile + S;
  bp->max_items = (n_total + kHistChunk - 1) / kHistChunk + S;
  const size_t per_seg = (size_t)(bp->places > 0 ? bp->places : 1) * kRadix * 4;
  size_t off = kHeaderBytes;
  bp->seg_done = off;
  off = round_up(off + S * 4);
  bp->seg_skew = off;
  off = round_up(off + S * (size_t)(bp->places > 0 ? bp->places : 1) * 4);
  bp->seg_hist = off;
  off = round_up(off + S * per_seg);
  bp->zero_end = off;
  bp->seg_bin_offsets = off;
  off = round_up(off + S * per_seg);
  bp->tile_base = off;
  off = round_up(off + (S + 1) * 4);
  bp->hist_base = off;
  off = round_up(off + (S + 1) * 4);
  bp->tile_seg = off;
  off = round_up(off + bp->max_tiles * 4);
  bp->hist_seg = off;
  off = round_up(off + bp->max_items * 4);
  const size_t slab = (size_t)bp->max_tiles * kRadix * 4;
  bp->status[0] = off;
  off = round_up(off + slab);
  bp->status[1] = off;
  off = round_up(off + (bp->places > 1 ? slab : 0));
  bp->alt_keys = off;
  off = round_up(off + (bp->places > 1 ? (size_t)n_total * (kb / 8) : 0));
  bp->alt_vals = off;
  off = round_up(off + (bp->places > 1 && bp->pairs ? (size_t)n_total * 4 : 0));
  bp->total = off;
  return OS_OK;
}

int run_batch(int key_type, const void* keys_in, void* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
              const uint64_t* seg_offsets, int64_t num_segments, uint64_t n_total, int begin_bit, int end_bit,
              void* ws, size_t ws_bytes, void* stream, int cfg_override = -1) {
  const bool pairs = vals_in != nullptr || vals_out != nullptr;
  if (pairs && (vals_in == nullptr || vals_out == nullptr)) return OS_ERR_INVALID_ARG;
  BatchPlan bp;
  int rc = make_batch_plan(key_type, n_total, num_segments, pairs ? 4 : 0, begin_bit, end_bit, &bp, cfg_override);
  if (rc != OS_OK) return rc;
  if (n_total == 0 || num_segments == 0) return OS_OK;
  const size_t kbytes = (size_t)n_total * (bp.key_bits / 8);
  const size_t vbytes = pairs ? (size_t)n_total * 4 : 0;
  if (!keys_in || !keys_out || !seg_offsets) return OS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(keys_in) % (bp.key_bits / 8) ||
      reinterpret_cast<uintptr_t>(keys_out) % (bp.key_bits / 8) || reinterpret_cast<uintptr_t>(seg_offsets) % 8)
    return OS_ERR_INVALID_ARG;
  if (pairs && (reinterpret_cast<uintptr_t>(vals_in) % 4 || reinterpret_cast<uintptr_t>(vals_out) % 4))
    return OS_ERR_INVALID_ARG;
  if (!ws || ws_bytes < bp.total) return OS_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % 16) return OS_ERR_INVALID_ARG;
  {
    const void* bufs[5] = {keys_in, keys_out, vals_in, vals_out, ws};
    const size_t sizes[5] = {kbytes, kbytes, vbytes, vbytes, bp.total};
    for (int i = 0; i < 5; ++i)
      for (int j = i + 1; j < 5; ++j)
        if (overlaps(bufs[i], sizes[i], bufs[j], sizes[j])) return OS_ERR_INVALID_ARG;
    if (overlaps(seg_offsets, ((size_t)num_segments + 1) * 8, keys_out, kbytes) ||
        overlaps(seg_offsets, ((size_t)num_segments + 1) * 8, vals_out, vbytes) ||
        overlaps(seg_offsets, ((size_t)num_segments + 1) * 8, ws, bp.total))
      return OS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  uint32_t* header = reinterpret_cast<uint32_t*>(w);

  if (bp.places == 0) {  // empty bit range: a plain copy
    if (cudaMemsetAsync(w, 0, 4, s) != cudaSuccess) return OS_ERR_CUDA;
    if (cudaMemcpyAsync(keys_out, keys_in, kbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return OS_ERR_CUDA;
    if (pairs && cudaMemcpyAsync(vals_out, vals_in, vbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return OS_ERR_CUDA;
    return OS_OK;
  }
  if (cudaMemsetAsync(w, 0, bp.zero_end, s) != cudaSuccess) return OS_ERR_CUDA;

  BatchArgs b{};
  b.keys_in = keys_in;
  b.keys_out = keys_out;
  b.vals_in = vals_in;
  b.vals_out = vals_out;
  b.seg_offsets = seg_offsets;
  b.num_segments = (uint32_t)num_segments;
  b.n_total = n_total;
  b.flip = is_float(key_type);
  b.num_places = bp.places;
  b.begin_bit = begin_bit;
  b.end_bit = end_bit;
  b.small_max = bp.small_max;
  b.tile_keys = bp.tile;
  b.hist_chunk = kHistChunk;
  b.max_tiles = (uint32_t)bp.max_tiles;
  b.max_items = (uint32_t)bp.max_items;
  b.tile_base = reinterpret_cast<uint32_t*>(w + bp.tile_base);
  b.tile_seg = reinterpret_cast<uint32_t*>(w + bp.tile_seg);
  b.hist_base = reinterpret_cast<uint32_t*>(w + bp.hist_base);
  b.hist_seg = reinterpret_cast<uint32_t*>(w + bp.hist_seg);
  b.totals = header + kTotalsWord;
  b.seg_done = reinterpret_cast<uint32_t*>(w + bp.seg_done);
  b.seg_hist = reinterpret_cast<uint32_t*>(w + bp.seg_hist);
  b.seg_bin_offsets = reinterpret_cast<uint32_t*>(w + bp.seg_bin_offsets);
  b.seg_skew = reinterpret_cast<uint32_t*>(w + bp.seg_skew);
  b.top_xor = signed_top_xor(key_type, begin_bit, end_bit);
  b.descending = is_descending(key_type) ? 1u : 0u;
  b.error = header;
  b.clear = reinterpret_cast<uint32_t*>(w + bp.status[0]);
  b.clear_words = bp.max_tiles * kRadix;

  int slot = prof_begin(2, -1, s);
  cudaError_t e = launch_batch_plan(b, s);
  prof_end(slot, s);
  if (e != cudaSuccess) return OS_ERR_CUDA;
  slot = prof_begin(0, -1, s);
  e = launch_batch_histogram(bp.key_bits, b, s);
  prof_end(slot, s);
  if (e != cudaSuccess) return OS_ERR_CUDA;
  slot = prof_begin(3, -1, s);
  e = launch_batch_local_sort(bp.key_bits, pairs, b, s);
  prof_end(slot, s);
  if (e != cudaSuccess) return OS_ERR_CUDA;

  void* alt_keys = w + bp.alt_keys;
  uint32_t* alt_vals = reinterpret_cast<uint32_t*>(w + bp.alt_vals);
  auto aligned16 = [](const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
  const void* src_k = keys_in;
  const uint32_t* src_v = vals_in;
  for (int pass = 0; pass < bp.places; ++pass) {
    const bool to_out = ((bp.places - 1 - pass) % 2) == 0;
    void* dst_k = to_out ? keys_out : alt_keys;
    uint32_t* dst_v = to_out ? vals_out : alt_vals;
    PassArgs a{};
    a.keys_in = src_k;
    a.keys_out = dst_k;
    a.vals_in = pairs ? src_v : nullptr;
    a.vals_out = pairs ? dst_v : nullptr;
    a.n = (uint32_t)n_total;
    a.num_tiles = (uint32_t)bp.max_tiles;
    a.shift = begin_bit + kRadixBits * pass;
    const int width = end_bit - a.shift < kRadixBits ? end_bit - a.shift : kRadixBits;
    a.mask = (1u << width) - 1u;
    a.flip_in = is_float(key_type) && pass == 0;
    a.flip_out = is_float(key_type) && pass == bp.places - 1;
    a.use_bulk = aligned16(src_k) && (!pairs || aligned16(src_v));
    a.bin_offsets = b.seg_bin_offsets + pass * kRadix;
    a.offsets_stride = (uint32_t)bp.places * kRadix;
    a.status = reinterpret_cast<uint32_t*>(w + bp.status[pass & 1]);
    a.status_clear = pass + 1 < bp.places ? reinterpret_cast<uint32_t*>(w + bp.status[(pass + 1) & 1]) : nullptr;
    a.status_clear_rows = (uint32_t)bp.max_tiles;  // every tile clears its own row
    a.tile_counter = header + kTileCounterWord + pass % 8;
    a.error = header;
    a.spin_limit = bp.spin_limit;
    a.fault_tile = bp.fault_tile;
    a.seg_offsets = seg_offsets;
    a.tile_base = b.tile_base;
    a.tile_seg = b.tile_seg;
    a.total_tiles = b.totals;
    a.skew_flags = b.seg_skew + pass;
    a.skew_stride = (uint32_t)bp.places;
    a.digit_xor = (pass == bp.places - 1 ? b.top_xor : 0u) ^ (b.descending ? a.mask : 0u);
    slot = prof_begin(1, pass, s);
    e = launch_binning(bp.key_bits, pairs, bp.cfg, a, s);
    prof_end(slot, s);
    if (e != cudaSuccess) return OS_ERR_CUDA;
    src_k = dst_k;
    src_v = dst_v;
  }
  return OS_OK;
}

}  // namespace

// The single-array sort on a workspace the caller already has (used by the
// entry point that takes its scratch from static device memory).
int sort_on_workspace(int key_type, const void* keys_in, void* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                      uint64_t n, int begin_bit, int end_bit, void* ws, size_t ws_bytes, void* stream) {
  return run_sort(key_type, keys_in, keys_out, vals_in, vals_out, n, begin_bit, end_bit, ws, ws_bytes, stream);
}

}  // namespace onesweep

using namespace onesweep;

extern "C" {

size_t os_sort_workspace_bytes(int key_type, uint64_t n, int value_bytes, int begin_bit, int end_bit) {
  Plan plan;
  if (make_plan(key_type, n, value_bytes, begin_bit, end_bit, &plan) != OS_OK) return 0;
  return plan.layout.total_bytes;
}

int os_sort_workspace_layout(int key_type, uint64_t n, int value_bytes, int begin_bit, int end_bit,
                             os_workspace_layout* layout) {
  if (!layout) return OS_ERR_INVALID_ARG;
  Plan plan;
  int rc = make_plan(key_type, n, value_bytes, begin_bit, end_bit, &plan);
  if (rc != OS_OK) return rc;
  *layout = plan.layout;
  return OS_OK;
}

int os_sort_keys(int key_type, const void* keys_in, void* keys_out, uint64_t n, int begin_bit, int end_bit,
                 void* ws, size_t ws_bytes, void* stream) {
  return run_sort(key_type, keys_in, keys_out, nullptr, nullptr, n, begin_bit, end_bit, ws, ws_bytes, stream);
}

int os_sort_pairs(int key_type, const void* keys_in, void* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                  uint64_t n, int begin_bit, int end_bit, void* ws, size_t ws_bytes, void* stream) {
  if (!vals_in || !vals_out) return OS_ERR_INVALID_ARG;
  return run_sort(key_type, keys_in, keys_out, vals_in, vals_out, n, begin_bit, end_bit, ws, ws_bytes, stream);
}

size_t os_sort_batch_workspace_bytes(int key_type, uint64_t n_total, int num_segments, int value_bytes,
                                     int begin_bit, int end_bit) {
  BatchPlan bp;
  if (make_batch_plan(key_type, n_total, num_segments, value_bytes, begin_bit, end_bit, &bp) != OS_OK) return 0;
  return bp.total;
}

int os_sort_batch(int key_type, const void* keys_in, void* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                  const uint64_t* seg_offsets, int num_segments, uint64_t n_total, int begin_bit, int end_bit, void* ws,
                  size_t ws_bytes, void* stream) {
  return run_batch(key_type, keys_in, keys_out, vals_in, vals_out, seg_offsets, num_segments, n_total, begin_bit,
                   end_bit, ws, ws_bytes, stream);
}

// The caller's binning variant (-1: the process-wide one) and digit width,
// or an error.
static int option_config(const os_sort_options* opt, int* cfg, int* radix_bits) {
  *cfg = -1;
  *radix_bits = 0;
  if (!opt) return OS_OK;
  if (opt->tile_config < -1 || opt->tile_config >= kTileConfigs) return OS_ERR_INVALID_ARG;
  if (opt->radix_bits != 0 && (opt->radix_bits < (uint32_t)kMinRadixBits || opt->radix_bits > (uint32_t)kRadixBits))
    return OS_ERR_INVALID_ARG;
  *cfg = opt->tile_config;
  if (opt->radix_bits != 0) *radix_bits = (int)opt->radix_bits;
  return OS_OK;
}

int os_sort_keys_ex(int key_type, const void* keys_in, void* keys_out, uint64_t n, int begin_bit, int end_bit,
                    void* ws, size_t ws_bytes, void* stream, const os_sort_options* opt) {
  int cfg;
  int rb;
  const int rc = option_config(opt, &cfg, &rb);
  if (rc != OS_OK) return rc;
  return run_sort(key_type, keys_in, keys_out, nullptr, nullptr, n, begin_bit, end_bit, ws, ws_bytes, stream, cfg,
                  rb);
}

int os_sort_pairs_ex(int key_type, const void* keys_in, void* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                     uint64_t n, int begin_bit, int end_bit, void* ws, size_t ws_bytes, void* stream,
                     const os_sort_options* opt) {
  if (!vals_in || !vals_out) return OS_ERR_INVALID_ARG;
  int cfg;
  int rb;
  const int rc = option_config(opt, &cfg, &rb);
  if (rc != OS_OK) return rc;
  return run_sort(key_type, keys_in, keys_out, vals_in, vals_out, n, begin_bit, end_bit, ws, ws_bytes, stream, cfg,
                  rb);
}

int os_sort_batch_ex(int key_type, const void* keys_in, void* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                     const uint64_t* seg_offsets, int num_segments, uint64_t n_total, int begin_bit, int end_bit,
                     void* ws, size_t ws_bytes, void* stream, const os_sort_options* opt) {
  int cfg;
  int rb;
  const int rc = option_config(opt, &cfg, &rb);
  if (rc != OS_OK) return rc;
  if (rb != 0 && rb != kRadixBits) return OS_ERR_INVALID_ARG;  // batches bin 8-bit digits
  return run_batch(key_type, keys_in, keys_out, vals_in, vals_out, seg_offsets, num_segments, n_total, begin_bit,
                   end_bit, ws, ws_bytes, stream, cfg);
}

int os_digit_histograms(int key_type, const void* keys_in, uint64_t n, int begin_bit, int end_bit,
                        uint32_t* hist_out, uint32_t* offsets_out, void* ws, size_t ws_bytes, void* stream) {
  Plan plan;
  int rc = make_plan(key_type, n, 0, begin_bit, end_bit, &plan);
  if (rc != OS_OK) return rc;
  if (!ws || ws_bytes < plan.layout.total_bytes) return OS_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % 16) return OS_ERR_INVALID_ARG;
  if (n > 0 && !keys_in) return OS_ERR_INVALID_ARG;
  if (n > 0 && reinterpret_cast<uintptr_t>(keys_in) % (plan.key_bits / 8)) return OS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  const size_t bytes = (size_t)plan.places * kRadix * 4;
  if (plan.places == 0) return OS_OK;
  // bin offsets are zeroed too, so n == 0 yields all-zero offsets
  if (cudaMemsetAsync(w, 0, plan.layout.bin_offset_offset + bytes, s) != cudaSuccess) return OS_ERR_CUDA;
  if (n > 0) {
    rc = run_histogram(plan, key_type, keys_in, n, begin_bit, end_bit, w, false, s);
    if (rc != OS_OK) return rc;
  }
  if (hist_out && cudaMemcpyAsync(hist_out, w + plan.layout.histogram_offset, bytes, cudaMemcpyDeviceToDevice, s) !=
                      cudaSuccess)
    return OS_ERR_CUDA;
  if (offsets_out && cudaMemcpyAsync(offsets_out, w + plan.layout.bin_offset_offset, bytes,
                                     cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return OS_ERR_CUDA;
  return OS_OK;
}

int os_workspace_status(const void* ws, void* stream) {
  if (!ws) return OS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return OS_ERR_CUDA;
  uint32_t word = 0;
  if (cudaMemcpy(&word, ws, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return OS_ERR_CUDA;
  if (word & kErrBadSegments) return OS_ERR_INVALID_ARG;
  if (word & kErrTimeout) return OS_ERR_TIMEOUT;
  return OS_OK;
}

const char* os_status_string(int status) {
  switch (status) {
    case OS_OK: return "ok";
    case OS_ERR_INVALID_ARG: return "invalid argument";
    case OS_ERR_TOO_LARGE: return "too many keys (n must be below 2^32)";
    case OS_ERR_WORKSPACE: return "workspace missing or too small";
    case OS_ERR_CUDA: return "CUDA error";
    case OS_ERR_TIMEOUT: return "chained-scan look-back wait ran past its limit";
    case OS_ERR_SCRATCH_LIMIT: return "sort too large for the fixed 16 MiB scratch of os_sort_noalloc";
    default: return "unknown status";
  }
}

int os_profile_start(int capacity) {
  std::lock_guard<std::mutex> lock(g_prof_mutex);
  if (g_prof || capacity <= 0) return OS_ERR_INVALID_ARG;
  ProfiledLaunch* p = new ProfiledLaunch[capacity];
  for (int i = 0; i < capacity; ++i) {
    if (cudaEventCreate(&p[i].start) != cudaSuccess || cudaEventCreate(&p[i].stop) != cudaSuccess) {
      for (int j = 0; j <= i; ++j) {
        cudaEventDestroy(p[j].start);
        cudaEventDestroy(p[j].stop);
      }
      delete[] p;
      return OS_ERR_CUDA;
    }
  }
  g_prof = p;
  g_prof_capacity = capacity;
  g_prof_used = 0;
  g_prof_seen = 0;
  g_prof_on.store(true, std::memory_order_release);
  return OS_OK;
}

int os_profile_stop(os_launch_time* out, int max, int* count) {
  std::lock_guard<std::mutex> lock(g_prof_mutex);
  if (!g_prof) return OS_ERR_INVALID_ARG;
  g_prof_on.store(false, std::memory_order_release);
  int rc = OS_OK;
  for (int i = 0; i < g_prof_used; ++i) {
    float ms = 0.f;
    if (cudaEventSynchronize(g_prof[i].stop) != cudaSuccess ||
        cudaEventElapsedTime(&ms, g_prof[i].start, g_prof[i].stop) != cudaSuccess)
      rc = OS_ERR_CUDA;
    if (out && i < max) out[i] = os_launch_time{g_prof[i].kernel, g_prof[i].pass, ms};
  }
  if (count) *count = g_prof_seen;
  for (int i = 0; i < g_prof_capacity; ++i) {
    cudaEventDestroy(g_prof[i].start);
    cudaEventDestroy(g_prof[i].stop);
  }
  delete[] g_prof;
  g_prof = nullptr;
  g_prof_capacity = g_prof_used = g_prof_seen = 0;
  return rc;
}

#define OS_STR2(x) #x
#define OS_STR(x) OS_STR2(x)
const char* os_build_info(void) { return "cuda_arch_list=" OS_STR(__CUDA_ARCH_LIST__); }
#undef OS_STR
#undef OS_STR2

int os_num_tile_configs(void) { return kTileConfigs; }

int os_tile_config_keys(int key_bits, int value_bytes, int cfg) {
  if ((key_bits != 32 && key_bits != 64) || (value_bytes != 0 && value_bytes != 4) || cfg < 0 ||
      cfg >= kTileConfigs)
    return 0;
  return (int)tile_keys_for(key_bits, value_bytes == 4, cfg);
}

int os_set_tile_config(int key_bits, int value_bytes, int cfg) {
  if ((key_bits != 32 && key_bits != 64) || (value_bytes != 0 && value_bytes != 4) || cfg < 0 ||
      cfg >= kTileConfigs)
    return OS_ERR_INVALID_ARG;
  for (int b = 0; b < kSizeBuckets; ++b) set_tile_cfg(key_bits, value_bytes == 4, b, cfg);
  return OS_OK;
}

int os_get_tile_config(int key_bits, int value_bytes) {
  if ((key_bits != 32 && key_bits != 64) || (value_bytes != 0 && value_bytes != 4)) return -1;
  return get_tile_cfg(key_bits, value_bytes == 4, kSizeBuckets - 1);
}

int os_num_size_buckets(void) { return kSizeBuckets; }

int os_size_bucket(uint64_t n) { return size_bucket(n); }

int os_set_tile_config_bucket(int key_bits, int value_bytes, int bucket, int cfg) {
  if ((key_bits != 32 && key_bits != 64) || (value_bytes != 0 && value_bytes != 4) || cfg < 0 ||
      cfg >= kTileConfigs || bucket < 0 || bucket >= kSizeBuckets)
    return OS_ERR_INVALID_ARG;
  set_tile_cfg(key_bits, value_bytes == 4, bucket, cfg);
  return OS_OK;
}

int os_get_tile_config_bucket(int key_bits, int value_bytes, int bucket) {
  if ((key_bits != 32 && key_bits != 64) || (value_bytes != 0 && value_bytes != 4) || bucket < 0 ||
      bucket >= kSizeBuckets)
    return -1;
  return get_tile_cfg(key_bits, value_bytes == 4, bucket);
}

int os_set_radix_bits_bucket(int key_bits, int value_bytes, int bucket, int radix_bits) {
  if ((key_bits != 32 && key_bits != 64) || (value_bytes != 0 && value_bytes != 4) || bucket < 0 ||
      bucket >= kSizeBuckets || radix_bits < kMinRadixBits || radix_bits > kRadixBits)
    return OS_ERR_INVALID_ARG;
  g_radix_bits[key_bits == 64][value_bytes == 4][bucket].store(radix_bits, std::memory_order_relaxed);
  return OS_OK;
}

int os_get_radix_bits_bucket(int key_bits, int value_bytes, int bucket) {
  if ((key_bits != 32 && key_bits != 64) || (value_bytes != 0 && value_bytes != 4) || bucket < 0 ||
      bucket >= kSizeBuckets)
    return -1;
  return get_radix_bits(key_bits, value_bytes == 4, bucket);
}

void os_debug_set_lookback_fault(int64_t tile, uint32_t spin_limit) {
  g_fault_tile.store(tile < 0 ? -1 : tile, std::memory_order_relaxed);
  g_spin_limit.store(spin_limit == 0 ? kDefaultSpinLimit : spin_limit, std::memory_order_relaxed);
}

uint64_t os_debug_set_strip_keys(uint64_t keys) {
  if (keys == 0 || keys > kStripKeys) keys = kStripKeys;
  if (keys < kMinStripKeys) keys = kMinStripKeys;
  g_strip_keys.store(keys, std::memory_order_relaxed);
  return keys;
}

}  // extern "C"
