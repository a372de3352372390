// batched.cu - persistent launches over the pair convolutions of many cells of unequal grid
// sides, k-meshes and band counts (V_x of Sec. II C for every cell of a batch).
//
// Each CTA takes work items from a global counter (largest first, as the host sorts them)
// until its list is exhausted; an item is (cell, k'-split, k, owner tile).  The items are
// split in two lists by the pipeline their side runs, each with its own persistent kernel:
//   * staged-partner items (sides 8, 12, 16, 18, 20; pairconv_tma.cuh): the partner orbitals
//     stream in by TMA from the cell's tensor map into two stage buffers, the owner orbital
//     and the accumulators stay in Tensor Memory.  512 threads; per cell the pencil layout
//     LayoutOne (one pencil per thread) or LayoutSeq (two), as the autotuner chose
//     (BatchCell::layout); 12^3 cells in LayoutOne, whose four owner slots need 576 threads,
//     form a third list with a kernel of its own;
//   * pencil-load items (side 24; pairconv_c64.cuh): orbitals are read as pencils through L1,
//     in the one-pencil form (18 warps, the single-cell default) or the ragged 12-warp form.
//     That kernel keeps only its own shared-memory footprint so that L1 keeps the rest of the
//     SM's storage: with the staged kernel's 208 KB of shared memory reserved, its 24^3 items
//     ran 37% slower.
// The two kernels may run on two streams at once: each takes every SM it can get, and the SMs
// the one finishing first frees go to the other.  Warps beyond an item's layout only take part
// in the block barriers.  One CTA per SM holds all 512 TMEM columns for the whole launch; the
// stage barriers' phases carry over from item to item.
#include "launch.cuh"

namespace hse {

namespace {

constexpr int kStagedThreads = 512;

template <int n>
using SeqS = GeoS<n, LayoutSeq<n>>;
template <int n>
using OneS = GeoS<n, LayoutOne<n>>;

static_assert(LayoutOne<20>::THREADS <= kStagedThreads && LayoutOne<8>::THREADS <= kStagedThreads &&
                  LayoutOne<16>::THREADS <= kStagedThreads &&
                  LayoutSeq<12>::THREADS <= kStagedThreads && LayoutOne<18>::THREADS <= kStagedThreads,
              "staged batched block too small for a side's layout");
static_assert(LayoutSeq<8>::THREADS <= kStagedThreads && LayoutSeq<16>::THREADS <= kStagedThreads &&
                  LayoutSeq<18>::THREADS <= kStagedThreads && LayoutSeq<20>::THREADS <= kStagedThreads,
              "staged batched block too small for a side's alternative layout");
static_assert(OneS<8>::FITS && SeqS<12>::FITS && OneS<16>::FITS && OneS<18>::FITS && OneS<20>::FITS &&
                  SeqS<8>::FITS && SeqS<16>::FITS && SeqS<18>::FITS && SeqS<20>::FITS,
              "staged layouts of the batched kernel must fit");

// One staged item as a call of its own: each side's pipeline gets the whole register budget
// instead of sharing one allocation with the other sides' inlined pipelines.  pa: the cell's
// launch arguments copied to shared memory; tmap: its tensor map (global memory).
template <int n, int MODE, template <int> class L>
__device__ __noinline__ bool staged_call(const PairArgs& pa, const CUtensorMap* tmap, int item, char* sbase,
                                         uint32_t tbase, StagedShared& sh, uint32_t& ph0, uint32_t& ph1, bool on) {
  return staged_item<n, MODE, L>(pa, tmap, item, sbase, tbase, sh, ph0, ph1, on);
}

// The cell's launch arguments into shared memory before an item (the item reads them many
// times; from the cell table in global memory every field would be a load that the
// register-bound pipelines cannot keep).  Every thread calls this; it synchronises the block.
__device__ __forceinline__ void load_cell_args(PairArgs* dst, const PairArgs& src) {
  static_assert(sizeof(PairArgs) % 8 == 0, "PairArgs copies as 8-byte words");
  const uint64_t* s = reinterpret_cast<const uint64_t*>(&src);
  uint64_t* d = reinterpret_cast<uint64_t*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(PairArgs) / 8); i += blockDim.x) d[i] = s[i];
  __syncthreads();
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
  __shared__ __align__(16) PairArgs pa_sh;
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
    load_cell_args(&pa_sh, c.pa);
    bool ok = true;
#define HSE_STAGED_CASE(N)                                                                              \
  case N:                                                                                               \
    ok = c.layout ? staged_call<N, MODE, LayoutSeq>(pa_sh, &c.tmap, wi.item, sbase, tbase, sh, ph0, ph1, \
                                                    warp < LayoutSeq<N>::WARPS)                          \
                  : staged_call<N, MODE, LayoutOne>(pa_sh, &c.tmap, wi.item, sbase, tbase, sh, ph0, ph1, \
                                                    warp < LayoutOne<N>::WARPS);                         \
    break;
    switch (c.n) {
      HSE_STAGED_CASE(8)
      case 12:
        ok = staged_call<12, MODE, LayoutSeq>(pa_sh, &c.tmap, wi.item, sbase, tbase, sh, ph0, ph1,
                                              warp < LayoutSeq<12>::WARPS);
        break;
      HSE_STAGED_CASE(16)
      HSE_STAGED_CASE(18)
      HSE_STAGED_CASE(20)
      default: break;  // the host puts only the sides above in this list
    }
#undef HSE_STAGED_CASE
    if (!ok) break;  // a bounded wait expired (uniform: read after a block barrier)
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(tbase, 512);
}

// The 12^3 items in LayoutOne (four owner slots of 144 threads, 576 threads): a kernel of its
// own, since the 512-thread staged kernel can only run 12^3 in LayoutSeq.
template <int MODE>
__global__ void __launch_bounds__(LayoutOne<12>::THREADS, 1) pairconv_batched_staged12_kernel(const BatchArgs b) {
  extern __shared__ __align__(128) float4 smem4[];
  __shared__ uint32_t tmem_base_sh;
  __shared__ StagedShared sh;
  __shared__ int next_sh;
  __shared__ __align__(16) PairArgs pa_sh;
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
    load_cell_args(&pa_sh, c.pa);
    const bool ok = c.n == 12 ? staged_item<12, MODE, LayoutOne>(pa_sh, &c.tmap, wi.item, sbase, tbase, sh, ph0, ph1,
                                                                 true)
                              : true;  // the host puts only 12^3 cells in this list
    if (!ok) break;
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(tbase, 512);
}

// PPT, TS: the pencil layout of the 24^3 items (one pencil per thread on 576 threads, or the
// ragged form on 384).
// BLK: the orbital layout of every cell in the list as a compile-time constant (1: all read
// pencil-blocked copies), or -1 (each cell's PairArgs::blk).
template <int MODE, int PPT, int TS, int BLK>
__global__ void __launch_bounds__(GeoP<24, PPT, TS>::THREADS, 1) pairconv_batched_pencil_kernel(const BatchArgs b) {
  extern __shared__ __align__(16) float4 smem4[];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int next_sh;
  __shared__ __align__(16) PairArgs pa_sh;
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
    load_cell_args(&pa_sh, c.pa);
    switch (c.n) {
      case 24:
        pairconv_item<24, MODE, PPT, TS, false, BLK>(pa_sh, wi.item, smem4, tbase, warp < GeoP<24, PPT, TS>::WARPS);
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
constexpr size_t kStagedSmem =
    max_c(max_c(max_c(OneS<8>::SMEM_REQUEST, SeqS<12>::SMEM_REQUEST), max_c(OneS<16>::SMEM_REQUEST, OneS<18>::SMEM_REQUEST)),
          max_c(max_c(OneS<20>::SMEM_REQUEST, SeqS<8>::SMEM_REQUEST),
                max_c(max_c(SeqS<16>::SMEM_REQUEST, SeqS<18>::SMEM_REQUEST), SeqS<20>::SMEM_REQUEST)));
// >= 118784: a second CTA (which would need TMEM too) never fits
constexpr size_t kPencilSmem = max_c(Geo<24>::SMEM_BYTES, (size_t)118784);
constexpr size_t kStaged12Smem = OneS<12>::SMEM_REQUEST;
static_assert(OneS<12>::FITS, "12^3 LayoutOne must fit its batched kernel");

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

template <int PPT, int TS, int BLK>
cudaError_t launch_pencil_list(const BatchArgs& pencil, int sms, cudaStream_t stream) {
  static bool done[64] = {};
  cudaError_t err = set_smem(pairconv_batched_pencil_kernel<MODE_APPLY, PPT, TS, BLK>, kPencilSmem, done);
  if (err != cudaSuccess) return err;
  pairconv_batched_pencil_kernel<MODE_APPLY, PPT, TS, BLK>
      <<<sms < pencil.nitems ? sms : pencil.nitems, GeoP<24, PPT, TS>::THREADS, kPencilSmem, stream>>>(pencil);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pairconv_batched(const BatchArgs& staged, const BatchArgs& staged12, const BatchArgs& pencil, int sms,
                                    int pencil_layout, bool pencil_blocked, cudaStream_t stream, cudaStream_t side,
                                    cudaEvent_t fork, cudaEvent_t join) {
  static bool done_s[64] = {}, done_12[64] = {};
  cudaError_t err = set_smem(pairconv_batched_staged_kernel<MODE_APPLY>, kStagedSmem, done_s);
  if (err == cudaSuccess) err = set_smem(pairconv_batched_staged12_kernel<MODE_APPLY>, kStaged12Smem, done_12);
  if (err != cudaSuccess) return err;
  const bool both = pencil.nitems > 0 && (staged.nitems > 0 || staged12.nitems > 0);
  const bool fork_side = both && side && fork && join;
  // the pencil-load list first: its 24^3 items are the longest; the staged list on the side
  // stream (when given) starts on the SMs the pencil kernel leaves and takes over its tail
  cudaStream_t s2 = stream;
  if (fork_side) {
    err = cudaEventRecord(fork, stream);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(side, fork, 0);
    if (err != cudaSuccess) return err;
    s2 = side;
  }
  if (pencil.nitems > 0) {
    if (pencil_layout == kPencilRagged)
      err = launch_pencil_list<2, kRaggedThreads, -1>(pencil, sms, stream);
    else  // one pencil per thread: the layout fixed at compile time where every cell is blocked
      err = pencil_blocked ? launch_pencil_list<1, Geo<24>::NN, 1>(pencil, sms, stream)
                           : launch_pencil_list<1, Geo<24>::NN, -1>(pencil, sms, stream);
    if (err != cudaSuccess) return err;
  }
  if (staged.nitems > 0) {
    pairconv_batched_staged_kernel<MODE_APPLY>
        <<<sms < staged.nitems ? sms : staged.nitems, kStagedThreads, kStagedSmem, s2>>>(staged);
    count_launch();
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (staged12.nitems > 0) {  // after the staged list, on its stream
    pairconv_batched_staged12_kernel<MODE_APPLY>
        <<<sms < staged12.nitems ? sms : staged12.nitems, LayoutOne<12>::THREADS, kStaged12Smem, s2>>>(staged12);
    count_launch();
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (fork_side) {
    err = cudaEventRecord(join, side);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(stream, join, 0);
  }
  return err;
}

}  // namespace hse
