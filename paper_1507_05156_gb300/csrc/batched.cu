// batched.cu - persistent launches over the pair convolutions of many cells of unequal grid
// sides, k-meshes and band counts (V_x of Sec. II C for every cell of a batch).
//
// Each CTA takes work items from a global counter (largest first, as the host sorts them)
// until its list is exhausted; an item is (cell, k'-split, k, owner tile).  The items are
// split in two lists by the pipeline their side runs, each with its own persistent kernel:
//   * staged-partner items (sides 8, 12, 16, 18, 20; pairconv_tma.cuh): the partner orbitals
//     stream in by TMA from the cell's tensor map into two stage buffers, the owner orbital
//     and the accumulators stay in Tensor Memory.  512 threads (8^3 with eight owner slots of
//     one pencil per thread);
//   * pencil-load items (side 24; pairconv_c64.cuh; in its ragged 12-warp form, 384 threads):
//     orbitals are read as pencils
//     through L1.  That kernel keeps only its own shared-memory footprint so that L1 keeps
//     the rest of the SM's storage: with the staged kernel's 208 KB of shared memory
//     reserved, its 24^3 items ran 37% slower.
// Warps beyond an item's layout only take part in the block barriers.  One CTA per SM holds
// all 512 TMEM columns for the whole launch; the stage barriers' phases carry over from item
// to item.
#include "launch.cuh"

namespace hse {

namespace {

constexpr int kStagedThreads = 512;
constexpr int kPencilThreads = kRaggedThreads;  // the ragged 24^3 form (12 warps)

template <int n>
using SeqS = GeoS<n, LayoutSeq<n>>;
template <int n>
using OneS = GeoS<n, LayoutOne<n>>;

static_assert(LayoutOne<20>::THREADS <= kStagedThreads && LayoutOne<8>::THREADS <= kStagedThreads &&
                  LayoutOne<16>::THREADS <= kStagedThreads &&
                  LayoutSeq<12>::THREADS <= kStagedThreads && LayoutOne<18>::THREADS <= kStagedThreads,
              "staged batched block too small for a side's layout");
static_assert(GeoP<24, 2, kRaggedThreads>::THREADS <= kPencilThreads,
              "pencil-load batched block too small");
static_assert(OneS<8>::FITS && SeqS<12>::FITS && OneS<16>::FITS && OneS<18>::FITS && OneS<20>::FITS,
              "staged layouts of the batched kernel must fit");

// One staged item as a call of its own: each side's pipeline gets the whole register budget
// instead of sharing one allocation with the other sides' inlined pipelines.
template <int n, int MODE, template <int> class L>
__device__ __noinline__ bool staged_call(const BatchCell& c, int item, char* sbase, uint32_t tbase, StagedShared& sh,
                                         uint32_t& ph0, uint32_t& ph1, bool on) {
  return staged_item<n, MODE, L>(c.pa, &c.tmap, item, sbase, tbase, sh, ph0, ph1, on);
}

// Next item of this CTA (block-uniform), or -1 when the list is exhausted.
__device__ __forceinline__ int next_item(const BatchArgs& b, int* next_sh) {
  if (threadIdx.x == 0) *next_sh = atomicAdd(b.counter, 1);
  __syncthreads();
  const int it = *next_sh;
  __syncthreads();  // every thread has read next_sh before it is overwritten
  return it < b.nitems ? it : -1;
}

template <int MODE>
__global__ void __launch_bounds__(kStagedThreads, 1) pairconv_batched_staged_kernel(const BatchArgs b) {
  extern __shared__ __align__(128) float4 smem4[];
  __shared__ uint32_t tmem_base_sh;
  __shared__ StagedShared sh;
  __shared__ int next_sh;
  char* sbase = staged_smem_base(smem4, b.status);
  if (!sbase) return;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(&sh.mbar[0], 1);
    mbar_init(&sh.mbar[1], 1);
    sh.abort = 0;
    mbar_fence_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base_sh, 512);
    tmem_relinquish();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tbase = tmem_base_sh;
  uint32_t ph0 = 0, ph1 = 0;
  for (;;) {
    const int it = next_item(b, &next_sh);
    if (it < 0) break;
    const BatchItem wi = b.items[it];
    const BatchCell& c = b.cells[wi.cell];
    bool ok = true;
    switch (c.n) {
      case 8: ok = staged_call<8, MODE, LayoutOne>(c, wi.item, sbase, tbase, sh, ph0, ph1, warp < LayoutOne<8>::WARPS); break;
      case 12: ok = staged_call<12, MODE, LayoutSeq>(c, wi.item, sbase, tbase, sh, ph0, ph1, warp < LayoutSeq<12>::WARPS); break;
      case 16: ok = staged_call<16, MODE, LayoutOne>(c, wi.item, sbase, tbase, sh, ph0, ph1, warp < LayoutOne<16>::WARPS); break;
      case 18: ok = staged_call<18, MODE, LayoutOne>(c, wi.item, sbase, tbase, sh, ph0, ph1, warp < LayoutOne<18>::WARPS); break;
      case 20: ok = staged_call<20, MODE, LayoutOne>(c, wi.item, sbase, tbase, sh, ph0, ph1, warp < LayoutOne<20>::WARPS); break;
      default: break;  // the host puts only the sides above in this list
    }
    if (!ok) break;  // a bounded wait expired (uniform: read after a block barrier)
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(tbase, 512);
}

template <int MODE>
__global__ void __launch_bounds__(kPencilThreads, 1) pairconv_batched_pencil_kernel(const BatchArgs b) {
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
    const int it = next_item(b, &next_sh);
    if (it < 0) break;
    const BatchItem wi = b.items[it];
    const BatchCell& c = b.cells[wi.cell];
    switch (c.n) {
      case 24:
        pairconv_item<24, MODE, 2, kRaggedThreads>(c.pa, wi.item, smem4, tbase,
                                                   warp < GeoP<24, 2, kRaggedThreads>::WARPS);
        break;
      default: break;  // the host puts only the sides above in this list
    }
    __syncthreads();  // the shared grid and TMEM rows are reused by the next item
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(tbase, 512);
}

constexpr size_t max_c(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kStagedSmem = max_c(max_c(max_c(OneS<8>::SMEM_REQUEST, SeqS<12>::SMEM_REQUEST), OneS<16>::SMEM_REQUEST),
                                     max_c(OneS<18>::SMEM_REQUEST, OneS<20>::SMEM_REQUEST));
// >= 118784: a second CTA (which would need TMEM too) never fits
constexpr size_t kPencilSmem = max_c(Geo<24>::SMEM_BYTES, (size_t)118784);

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes, bool* done) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!done[dev]) {
    cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (err != cudaSuccess) return err;
    done[dev] = true;
  }
  return cudaSuccess;
}

}  // namespace

bool batched_side_supported(int n) { return n == 8 || n == 12 || n == 16 || n == 18 || n == 20 || n == 24; }

bool batched_stage_geometry(int n, int* sp, int* box_rows) {
  switch (n) {
    case 8: *sp = StageGeo<8>::SP; *box_rows = StageGeo<8>::BR; return true;
    case 12: *sp = StageGeo<12>::SP; *box_rows = StageGeo<12>::BR; return true;
    case 16: *sp = StageGeo<16>::SP; *box_rows = StageGeo<16>::BR; return true;
    case 18: *sp = StageGeo<18>::SP; *box_rows = StageGeo<18>::BR; return true;
    case 20: *sp = StageGeo<20>::SP; *box_rows = StageGeo<20>::BR; return true;
    default: return false;
  }
}

cudaError_t launch_pairconv_batched(const BatchArgs& staged, const BatchArgs& pencil, int sms, cudaStream_t stream) {
  static bool done_s[64] = {}, done_p[64] = {};
  cudaError_t err = set_smem(pairconv_batched_staged_kernel<MODE_APPLY>, kStagedSmem, done_s);
  if (err == cudaSuccess) err = set_smem(pairconv_batched_pencil_kernel<MODE_APPLY>, kPencilSmem, done_p);
  if (err != cudaSuccess) return err;
  // the pencil-load list first: its 24^3 items are the longest, and the staged list's short
  // items fill the tail
  if (pencil.nitems > 0) {
    pairconv_batched_pencil_kernel<MODE_APPLY>
        <<<sms < pencil.nitems ? sms : pencil.nitems, kPencilThreads, kPencilSmem, stream>>>(pencil);
    count_launch();
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (staged.nitems > 0) {
    pairconv_batched_staged_kernel<MODE_APPLY>
        <<<sms < staged.nitems ? sms : staged.nitems, kStagedThreads, kStagedSmem, stream>>>(staged);
    count_launch();
    err = cudaGetLastError();
  }
  return err;
}

}  // namespace hse
