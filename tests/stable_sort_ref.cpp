// Cross-check for the oracle's sort: std::stable_sort of the indices by the
// sorted-on field of each key - the bits [begin, end) of the key's order
// bits (unsigned: the key itself; signed: sign bit inverted; float: the
// sign-flip, negative keys all bits inverted) - compared as unsigned
// integers. Test infrastructure only; built by tests/test_stable_sort_ref.py.
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <numeric>
#include <vector>

namespace {

template <typename U>
U order_bits(U k, int kind) {  // kind: 0 unsigned, 1 signed, 2 float
  const U sign = (U)1 << (sizeof(U) * 8 - 1);
  if (kind == 1) return k ^ sign;
  if (kind == 2) return (k & sign) ? (U)~k : (U)(k | sign);
  return k;
}

template <typename U>
void stable_perm(const U* keys, uint32_t* perm, size_t n, int begin, int end, int kind) {
  const int width = end - begin;
  const U mask = width >= (int)(sizeof(U) * 8) ? (U)~(U)0 : (U)(((U)1 << width) - 1);
  std::vector<U> field(n);
  for (size_t i = 0; i < n; ++i) field[i] = width == 0 ? 0 : (U)((order_bits(keys[i], kind) >> begin) & mask);
  std::vector<uint32_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0u);
  std::stable_sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) { return field[a] < field[b]; });
  std::copy(idx.begin(), idx.end(), perm);
}

}  // namespace

extern "C" {
void ref_stable_perm32(const uint32_t* keys, uint32_t* perm, size_t n, int begin, int end, int kind) {
  stable_perm<uint32_t>(keys, perm, n, begin, end, kind);
}
void ref_stable_perm64(const uint64_t* keys, uint32_t* perm, size_t n, int begin, int end, int kind) {
  stable_perm<uint64_t>(keys, perm, n, begin, end, kind);
}
}
