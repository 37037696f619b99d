// Instantiations of the digit-binning kernel: 32-bit keys, keys, float
// transform mode 3 (bit 0: sign-flip on load, bit 1: undo on store),
// one array.
#include "os_binning_ws.cuh"

namespace onesweep {

cudaError_t launch_binning32_keys_f3_single(int cfg, int rank, const PassArgs& a, cudaStream_t s) {
  return launch_binning_flip<32, false, 3, false>(a, s, cfg, rank);
}

}  // namespace onesweep
