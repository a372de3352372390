// Fused complex64 pair-convolution kernels, cubic grids 16^3 and 18^3.
#include "launch.cuh"

namespace hse {
cudaError_t launch_pairconv_c64_mid(int n, int mode, const PairArgs& args, int bps, cudaStream_t stream) {
  switch (n) {
    case 16: return launch_pairconv_c64_n<16>(mode, args, bps, stream);
    case 18: return launch_pairconv_c64_n<18>(mode, args, bps, stream);
    default: return cudaErrorInvalidValue;
  }
}

int occupancy_pairconv_c64_mid(int n, int mode, int bps) {
  switch (n) {
    case 16: return pairconv_occupancy_n<16>(mode, bps);
    case 18: return pairconv_occupancy_n<18>(mode, bps);
    default: return 0;
  }
}

bool pencil_load_pairconv_c64_mid(int n, int mode, int bps) {
  switch (n) {
    case 16: return pencil_load_n<16>(mode, bps);
    case 18: return pencil_load_n<18>(mode, bps);
    default: return true;
  }
}
}  // namespace hse
