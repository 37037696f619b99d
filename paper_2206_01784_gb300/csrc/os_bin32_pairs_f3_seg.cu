// Instantiations of the digit-binning kernel: 32-bit keys, pairs, float
// transform mode 3 (bit 0: sign-flip on load, bit 1: undo on store),
// segmented (batch) mode.
#include "os_binning_ws.cuh"

namespace onesweep {

cudaError_t launch_binning32_pairs_f3_seg(int cfg, int rank, const PassArgs& a, cudaStream_t s) {
  return launch_binning_flip<32, true, 3, true>(a, s, cfg, rank);
}

}  // namespace onesweep
