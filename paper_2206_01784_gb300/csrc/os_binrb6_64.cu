// Instantiations of the digit-binning kernel with 6-bit digits: 64-bit keys,
// keys only and pairs, every float transform mode, one array.
#include "os_binning_ws.cuh"

namespace onesweep {

cudaError_t launch_binning_rb6_64(bool pairs, int flip, const PassArgs& a, cudaStream_t s) {
  return launch_binning_rb_t<64, 6>(pairs, flip, a, s);
}

}  // namespace onesweep
