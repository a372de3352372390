// Fused complex64 pair-convolution kernels, cubic grid 24^3.
#include "launch.cuh"

namespace hse {
cudaError_t launch_pairconv_c64_24(int mode, const PairArgs& args, int bps, cudaStream_t stream) {
  return launch_pairconv_c64_n<24>(mode, args, bps, stream);
}

int occupancy_pairconv_c64_24(int mode, int bps) { return pairconv_occupancy_n<24>(mode, bps); }

bool pencil_load_pairconv_c64_24(int mode, int bps) { return pencil_load_n<24>(mode, bps); }
}  // namespace hse
