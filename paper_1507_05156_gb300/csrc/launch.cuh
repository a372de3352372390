// launch.cuh - internal launcher declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "pairconv_c64.cuh"
#include "staged_f64.cuh"

namespace hse {

void count_launch(int n = 1);

// Fused complex64 pair-convolution launch for a cubic grid of side n (one TU per size
// group keeps the build parallel).  Returns a cudaError_t.
cudaError_t launch_pairconv_c64(int n, int mode, const PairArgs& args, cudaStream_t stream);
bool pairconv_c64_supported(int n);

// One staged FP64 1-D transform pass along an axis of length L with element stride inner.
cudaError_t launch_staged_fft(int L, int dir, double2* work, size_t nbatch, int N, int inner, cudaStream_t stream);
bool staged_fft_supported(int L);

// Template body used by the per-size translation units.
template <int n>
cudaError_t launch_pairconv_c64_n(int mode, const PairArgs& args, cudaStream_t stream) {
  constexpr size_t smem = pairconv_smem_bytes<n>();
  constexpr int threads = slots_for(n) * n * n;
  const dim3 grid((unsigned)((size_t)args.nk * args.ntiles));
  cudaError_t err = cudaSuccess;
  switch (mode) {
#define HSE_PC_CASE(M)                                                                                     \
  case M: {                                                                                               \
    static bool attr_done[64] = {};                                                                       \
    int dev = 0;                                                                                          \
    cudaGetDevice(&dev);                                                                                  \
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;                                              \
    if (!attr_done[dev]) {                                                                                \
      err = cudaFuncSetAttribute(pairconv_c64_kernel<n, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)smem);                                                              \
      if (err != cudaSuccess) return err;                                                                 \
      attr_done[dev] = true;                                                                              \
    }                                                                                                     \
    pairconv_c64_kernel<n, M><<<grid, threads, smem, stream>>>(args);                                     \
    break;                                                                                                \
  }
    HSE_PC_CASE(MODE_APPLY)
    HSE_PC_CASE(MODE_ENERGY)
    HSE_PC_CASE(MODE_DOT)
    HSE_PC_CASE(MODE_OCC)
#undef HSE_PC_CASE
    default:
      return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace hse
