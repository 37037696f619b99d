// Instantiations of the digit-binning kernel for 32-bit keys (uint32, float32).
#include "os_binning.cuh"

namespace onesweep {

cudaError_t launch_binning32(bool pairs, bool match, const PassArgs& a, cudaStream_t s) {
  return pairs ? launch_binning_t<32, true>(a, s, match) : launch_binning_t<32, false>(a, s, match);
}

uint32_t binning_tile_keys32(bool pairs) {
  return pairs ? BinningConfig<32, true>::T : BinningConfig<32, false>::T;
}

}  // namespace onesweep
