// Fused complex64 pair-convolution kernels, cubic grid 24^3.
#include "launch.cuh"

namespace hse {
cudaError_t launch_pairconv_c64_24(int mode, const PairArgs& args, cudaStream_t stream) {
  return launch_pairconv_c64_n<24>(mode, args, stream);
}
}  // namespace hse
