// batched.cu - one persistent launch over the pair convolutions of many cells of unequal grid
// sides, k-meshes and band counts (V_x of Sec. II C for every cell of a batch).
//
// Each CTA takes work items from a global counter (largest first, as the host sorts them)
// until the list is exhausted; an item is (cell, k'-split, k, owner tile) and runs the pencil
// pipeline of pairconv_c64.cuh for that cell's grid side.  The block has the largest thread
// count of the sides present (smaller sides leave whole warps idle), the largest shared-memory
// grid, and all 512 TMEM columns, so one CTA runs per SM.
#include "launch.cuh"

namespace hse {

namespace {

constexpr int kBatchThreads = 288;  // max Geo<n>::THREADS over the batched sides

template <int MODE>
__global__ void __launch_bounds__(kBatchThreads, 1) pairconv_batched_kernel(const BatchArgs b) {
  extern __shared__ __align__(16) float4 smem4[];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int next_sh;
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    tmem_alloc(&tmem_base_sh, 512);
    tmem_relinquish();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tbase = tmem_base_sh;
  for (;;) {
    if (threadIdx.x == 0) next_sh = atomicAdd(b.counter, 1);
    __syncthreads();
    const int it = next_sh;
    __syncthreads();  // every thread has read next_sh before it is overwritten
    if (it >= b.nitems) break;
    const BatchItem wi = b.items[it];
    const BatchCell& c = b.cells[wi.cell];
    switch (c.n) {
      case 8: pairconv_item<8, MODE>(c.pa, wi.item, smem4, tbase, warp < Geo<8>::WARPS); break;
      case 12: pairconv_item<12, MODE>(c.pa, wi.item, smem4, tbase, warp < Geo<12>::WARPS); break;
      case 16: pairconv_item<16, MODE>(c.pa, wi.item, smem4, tbase, warp < Geo<16>::WARPS); break;
      case 18: pairconv_item<18, MODE>(c.pa, wi.item, smem4, tbase, warp < Geo<18>::WARPS); break;
      case 20: pairconv_item<20, MODE>(c.pa, wi.item, smem4, tbase, warp < Geo<20>::WARPS); break;
      case 24: pairconv_item<24, MODE>(c.pa, wi.item, smem4, tbase, warp < Geo<24>::WARPS); break;
      default: break;  // the host admits only the sides above
    }
    __syncthreads();  // the shared grid and TMEM rows are reused by the next item
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(tbase, 512);
}

constexpr size_t max_c(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kBatchSmem =
    max_c(max_c(max_c(Geo<8>::SMEM_BYTES, Geo<12>::SMEM_BYTES), max_c(Geo<16>::SMEM_BYTES, Geo<18>::SMEM_BYTES)),
          max_c(max_c(Geo<20>::SMEM_BYTES, Geo<24>::SMEM_BYTES), (size_t)118784));  // >= 118784: one CTA per SM

static_assert(Geo<24>::THREADS <= kBatchThreads && Geo<12>::THREADS <= kBatchThreads, "batch block too small");

}  // namespace

bool batched_side_supported(int n) { return n == 8 || n == 12 || n == 16 || n == 18 || n == 20 || n == 24; }

cudaError_t launch_pairconv_batched(const BatchArgs& b, int sms, cudaStream_t stream) {
  static bool attr_done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr_done[dev]) {
    cudaError_t err = cudaFuncSetAttribute(pairconv_batched_kernel<MODE_APPLY>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem);
    if (err != cudaSuccess) return err;
    attr_done[dev] = true;
  }
  const int grid = sms < b.nitems ? sms : b.nitems;
  if (grid <= 0) return cudaSuccess;
  pairconv_batched_kernel<MODE_APPLY><<<grid, kBatchThreads, kBatchSmem, stream>>>(b);
  count_launch();
  return cudaGetLastError();
}

}  // namespace hse
