// Instantiations of the digit-binning kernel: 64-bit keys, pairs, float
// transform mode 2 (bit 0: sign-flip on load, bit 1: undo on store),
// segmented (batch) mode.
#include "os_binning_ws.cuh"

namespace onesweep {

cudaError_t launch_binning64_pairs_f2_seg(int cfg, int rank, const PassArgs& a, cudaStream_t s) {
  return launch_binning_flip<64, true, 2, true>(a, s, cfg, rank);
}

}  // namespace onesweep
