// Instantiations of the digit-binning kernel for 64-bit keys (uint64, float64).
#include "os_binning.cuh"

namespace onesweep {

cudaError_t launch_binning64(bool pairs, bool match, const PassArgs& a, cudaStream_t s) {
  return pairs ? launch_binning_t<64, true>(a, s, match) : launch_binning_t<64, false>(a, s, match);
}

uint32_t binning_tile_keys64(bool pairs) {
  return pairs ? BinningConfig<64, true>::T : BinningConfig<64, false>::T;
}

}  // namespace onesweep
