// Instantiations of the digit-binning kernel: 64-bit keys, keys, float
// transform mode 0 (bit 0: sign-flip on load, bit 1: undo on store),
// segmented (batch) mode.
#include "os_binning_ws.cuh"

namespace onesweep {

cudaError_t launch_binning64_keys_f0_seg(int cfg, int rank, const PassArgs& a, cudaStream_t s) {
  return launch_binning_flip<64, false, 0, true>(a, s, cfg, rank);
}

}  // namespace onesweep
