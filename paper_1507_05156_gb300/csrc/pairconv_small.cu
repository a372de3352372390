// Fused complex64 pair-convolution kernels, cubic grids up to 12^3.
#include "launch.cuh"

namespace hse {
cudaError_t launch_pairconv_c64_small(int n, int mode, const PairArgs& args, int bps, cudaStream_t stream) {
  switch (n) {
    case 4: return launch_pairconv_c64_n<4>(mode, args, bps, stream);
    case 6: return launch_pairconv_c64_n<6>(mode, args, bps, stream);
    case 8: return launch_pairconv_c64_n<8>(mode, args, bps, stream);
    case 10: return launch_pairconv_c64_n<10>(mode, args, bps, stream);
    case 12: return launch_pairconv_c64_n<12>(mode, args, bps, stream);
    default: return cudaErrorInvalidValue;
  }
}

int occupancy_pairconv_c64_small(int n, int mode, int bps) {
  switch (n) {
    case 4: return pairconv_occupancy_n<4>(mode, bps);
    case 6: return pairconv_occupancy_n<6>(mode, bps);
    case 8: return pairconv_occupancy_n<8>(mode, bps);
    case 10: return pairconv_occupancy_n<10>(mode, bps);
    case 12: return pairconv_occupancy_n<12>(mode, bps);
    default: return 0;
  }
}

bool pencil_load_pairconv_c64_small(int n, int mode, int bps) {
  switch (n) {
    case 4: return pencil_load_n<4>(mode, bps);
    case 6: return pencil_load_n<6>(mode, bps);
    case 8: return pencil_load_n<8>(mode, bps);
    case 10: return pencil_load_n<10>(mode, bps);
    case 12: return pencil_load_n<12>(mode, bps);
    default: return true;
  }
}
}  // namespace hse
