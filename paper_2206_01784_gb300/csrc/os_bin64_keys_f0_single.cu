// Instantiations of the digit-binning kernel: 64-bit keys, keys, float
// transform mode 0 (bit 0: sign-flip on load, bit 1: undo on store),
// one array.
#include "os_binning_ws.cuh"

namespace onesweep {

cudaError_t launch_binning64_keys_f0_single(int cfg, int rank, const PassArgs& a, cudaStream_t s) {
  return launch_binning_flip<64, false, 0, false>(a, s, cfg, rank);
}

uint32_t binning_tile_keys64_keys(int cfg) { return tile_keys_t<64, false>(cfg); }

}  // namespace onesweep
