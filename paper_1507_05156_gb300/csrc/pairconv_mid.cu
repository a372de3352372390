// Fused complex64 pair-convolution kernels, cubic grids 15^3 to 18^3.
#include "launch.cuh"

namespace hse {
cudaError_t launch_pairconv_c64_mid(int n, int mode, const PairArgs& args, cudaStream_t stream) {
  switch (n) {
    case 15: return launch_pairconv_c64_n<15>(mode, args, stream);
    case 16: return launch_pairconv_c64_n<16>(mode, args, stream);
    case 18: return launch_pairconv_c64_n<18>(mode, args, stream);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace hse
