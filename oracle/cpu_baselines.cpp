// CPU baselines for the benchmark's comparison rows (arXiv 2206.01784 sorts on
// the GPU; these are the same problem on the host's cores).
//
// TEST AND BENCHMARK INFRASTRUCTURE, like the oracle beside it: only the test
// suite and the benchmark's CPU-baseline leg load this library; the product
// path never does, and it shares no code with the CUDA path. It is not the
// oracle either (the oracle is onesweep_oracle.c, plain and one key at a
// time); tests/test_cpu_baselines.py checks both routines here bit for bit
// against it.
//
//  - cpb_parallel_lsd: the LSD radix sort of Section 1 (stable counting sort
//    by 8-bit places, least significant first) spread over T host threads:
//    each thread counts the digits of its contiguous share of the input, the
//    (digit, thread) counts are prefix-summed in digit-major order, and each
//    thread scatters its share in input order - which keeps the sort stable;
//  - cpb_std_stable_sort: std::stable_sort of (ordered field, position) on one
//    thread, the library comparison sort.
//
// Key types and readings as the oracle's: unsigned keys as they are, signed
// keys with the sign bit inverted, IEEE keys by the sign-flip (negative keys
// inverted, others with the sign bit set), sorted on the field
// [begin_bit, end_bit) of those ordered bits; values follow their keys.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

enum { U32 = 0, U64 = 1, F32 = 2, F64 = 3, I32 = 4, I64 = 5 };

bool wide(int kt) { return kt == U64 || kt == F64 || kt == I64; }

template <typename K>
K ordered(int kt, K b) {
  constexpr int top = sizeof(K) * 8 - 1;
  const K sign = K(1) << top;
  if (kt == I32 || kt == I64) return b ^ sign;
  if (kt == F32 || kt == F64) return (b & sign) ? K(~b) : K(b | sign);
  return b;
}

template <typename K>
K unordered(int kt, K u) {
  constexpr int top = sizeof(K) * 8 - 1;
  const K sign = K(1) << top;
  if (kt == I32 || kt == I64) return u ^ sign;
  if (kt == F32 || kt == F64) return (u & sign) ? K(u & ~sign) : K(~u);
  return u;
}

template <typename K>
int parallel_lsd(int kt, const K* in, const uint32_t* vin, uint64_t n, int begin_bit, int end_bit, int threads,
                 K* out, uint32_t* vout) {
  const int places = end_bit > begin_bit ? (end_bit - begin_bit + 7) / 8 : 0;
  if (threads < 1) threads = 1;
  if ((uint64_t)threads > n / 4096 + 1) threads = (int)(n / 4096 + 1);
  std::vector<K> a(n), b(n);
  std::vector<uint32_t> va(vin ? n : 0), vb(vin ? n : 0);
  auto share = [&](int t, uint64_t* lo, uint64_t* hi) {
    *lo = n * (uint64_t)t / threads;
    *hi = n * (uint64_t)(t + 1) / threads;
  };
  auto run = [&](auto&& body) {
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(body, t);
    body(0);
    for (auto& th : pool) th.join();
  };
  run([&](int t) {
    uint64_t lo, hi;
    share(t, &lo, &hi);
    for (uint64_t i = lo; i < hi; ++i) a[i] = ordered<K>(kt, in[i]);
    if (vin) std::memcpy(va.data() + lo, vin + lo, (hi - lo) * 4);
  });
  std::vector<uint64_t> count((size_t)threads * 256), offset((size_t)threads * 256);
  for (int place = 0; place < places; ++place) {
    const int shift = begin_bit + 8 * place;
    const int width = std::min(8, end_bit - shift);
    const K mask = (K)((1u << width) - 1u);
    run([&](int t) {
      uint64_t lo, hi;
      share(t, &lo, &hi);
      uint64_t* c = count.data() + (size_t)t * 256;
      std::fill(c, c + 256, 0);
      for (uint64_t i = lo; i < hi; ++i) ++c[(a[i] >> shift) & mask];
    });
    uint64_t run_sum = 0;
    for (int d = 0; d < 256; ++d)
      for (int t = 0; t < threads; ++t) {
        offset[(size_t)t * 256 + d] = run_sum;
        run_sum += count[(size_t)t * 256 + d];
      }
    run([&](int t) {
      uint64_t lo, hi;
      share(t, &lo, &hi);
      uint64_t* o = offset.data() + (size_t)t * 256;
      for (uint64_t i = lo; i < hi; ++i) {
        const uint64_t dst = o[(a[i] >> shift) & mask]++;
        b[dst] = a[i];
        if (vin) vb[dst] = va[i];
      }
    });
    a.swap(b);
    va.swap(vb);
  }
  run([&](int t) {
    uint64_t lo, hi;
    share(t, &lo, &hi);
    for (uint64_t i = lo; i < hi; ++i) out[i] = unordered<K>(kt, a[i]);
    if (vin) std::memcpy(vout + lo, va.data() + lo, (hi - lo) * 4);
  });
  return 0;
}

template <typename K>
int std_stable(int kt, const K* in, const uint32_t* vin, uint64_t n, int begin_bit, int end_bit, K* out,
               uint32_t* vout) {
  const int w = end_bit - begin_bit;
  const K mask = w >= (int)(sizeof(K) * 8) ? K(~K(0)) : K((K(1) << w) - 1);
  std::vector<std::pair<K, uint32_t>> rec(n);
  for (uint64_t i = 0; i < n; ++i) rec[i] = {K((ordered<K>(kt, in[i]) >> begin_bit) & mask), (uint32_t)i};
  std::stable_sort(rec.begin(), rec.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  for (uint64_t i = 0; i < n; ++i) {
    out[i] = in[rec[i].second];
    if (vin) vout[i] = vin[rec[i].second];
  }
  return 0;
}

bool valid(int kt, int begin_bit, int end_bit, const void* vin, const void* vout) {
  const int bits = wide(kt) ? 64 : 32;
  if (kt < 0 || kt > 5 || begin_bit < 0 || end_bit > bits || begin_bit > end_bit) return false;
  return (vin == nullptr) == (vout == nullptr);
}

}  // namespace

extern "C" {

// Stable ascending sort on `threads` host threads. Returns 0, or -1 on bad arguments.
int cpb_parallel_lsd(int key_type, const void* keys_in, const uint32_t* vals_in, uint64_t n, int begin_bit,
                     int end_bit, int threads, void* keys_out, uint32_t* vals_out) {
  if (!valid(key_type, begin_bit, end_bit, vals_in, vals_out)) return -1;
  if (wide(key_type))
    return parallel_lsd<uint64_t>(key_type, (const uint64_t*)keys_in, vals_in, n, begin_bit, end_bit, threads,
                                  (uint64_t*)keys_out, vals_out);
  return parallel_lsd<uint32_t>(key_type, (const uint32_t*)keys_in, vals_in, n, begin_bit, end_bit, threads,
                                (uint32_t*)keys_out, vals_out);
}

// Stable ascending sort with std::stable_sort on one thread.
int cpb_std_stable_sort(int key_type, const void* keys_in, const uint32_t* vals_in, uint64_t n, int begin_bit,
                        int end_bit, void* keys_out, uint32_t* vals_out) {
  if (!valid(key_type, begin_bit, end_bit, vals_in, vals_out)) return -1;
  if (wide(key_type))
    return std_stable<uint64_t>(key_type, (const uint64_t*)keys_in, vals_in, n, begin_bit, end_bit,
                                (uint64_t*)keys_out, vals_out);
  return std_stable<uint32_t>(key_type, (const uint32_t*)keys_in, vals_in, n, begin_bit, end_bit,
                              (uint32_t*)keys_out, vals_out);
}

int cpb_hardware_threads(void) {
  const unsigned t = std::thread::hardware_concurrency();
  return t ? (int)t : 1;
}

}  // extern "C"
