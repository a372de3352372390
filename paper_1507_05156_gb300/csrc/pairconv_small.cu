// Fused complex64 pair-convolution kernels, cubic grids up to 12^3.
#include "launch.cuh"

namespace hse {
cudaError_t launch_pairconv_c64_small(int n, int mode, const PairArgs& args, cudaStream_t stream) {
  switch (n) {
    case 4: return launch_pairconv_c64_n<4>(mode, args, stream);
    case 6: return launch_pairconv_c64_n<6>(mode, args, stream);
    case 8: return launch_pairconv_c64_n<8>(mode, args, stream);
    case 10: return launch_pairconv_c64_n<10>(mode, args, stream);
    case 12: return launch_pairconv_c64_n<12>(mode, args, stream);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace hse
