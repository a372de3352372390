// launch.cuh - internal launcher declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "pairconv_c64.cuh"
#include "pairconv_tma.cuh"
#include "staged_f64.cuh"

namespace hse {

void count_launch(int n = 1);

// Kinetic term 1/2 |G + k + A|^2 on nk x nbands orbitals (kinetic.cu).
struct KinArgs {
  int n1, n2, n3, nk, nbands, ntiles;
  double b[9];          // reciprocal rows b1, b2, b3
  double A[3];          // vector potential (bohr^-1)
  const double* kpts;   // device [nk][3]
};
cudaError_t launch_kinetic_f64(const double2* u, double2* out, const KinArgs& a, cudaStream_t stream);

// Taylor-step accumulation and the electric current (tdks.cu).
struct CurArgs {
  int n1, n2, n3, nk, nbands;
  double b[9];          // reciprocal rows b1, b2, b3
  double A[3];          // vector potential (bohr^-1)
  const double* kpts;   // device [nk][3]
};
cudaError_t launch_taylor_accumulate(bool c128, const void* kin, const void* vx, const void* prev, const double* vloc,
                                     size_t N, void* term, void* out, size_t count, double s, cudaStream_t stream);
// v_H (device double [N]) of the orbitals' density; work: [N] double2 scratch.
cudaError_t launch_hartree(bool c128, const void* psi, const double* occ, const CurArgs& a, double spin_degeneracy,
                           double2* work, double* vh, cudaStream_t stream);
// J (device double[3]) from the orbitals psi [nk][nbands][N] and occupations [nk][nbands];
// work: [nk][nbands][N] double2 scratch, partial: [nk][nbands][3] double scratch.
cudaError_t launch_current(bool c128, const void* psi, const double* occ, const CurArgs& a, double2* work,
                           double* partial, double spin_degeneracy, double* J, cudaStream_t stream);

// Overlap matrices and Gram-Schmidt orthonormalisation in FP64 (ortho.cu).
constexpr int kStatusSingular = -8;  // HSE_ERR_SINGULAR
// S device [nk][nb][nb] double2: S[k][a][b] = dV sum_r conj(u_{a,k}) u_{b,k}
cudaError_t launch_overlap(bool c128, const void* u, int nk, int nb, size_t N, double dV, double2* S,
                           cudaStream_t stream);
// u [nk][nb][N] in place (two modified Gram-Schmidt passes); work: [nk][nb][N] double2
// scratch for complex64 orbitals (unused for complex128); status: the plan's status word.
cudaError_t launch_orthonormalize(bool c128, void* u, int nk, int nb, size_t N, double dV, double2* work, int* status,
                                  cudaStream_t stream);

// Fused complex64 pair-convolution launch for a cubic grid of side n (one TU per size
// group keeps the build parallel).  Returns a cudaError_t.
cudaError_t launch_pairconv_c64(int n, int mode, const PairArgs& args, int blocks_per_sm, cudaStream_t stream);
bool pairconv_c64_supported(int n);
cudaError_t launch_kinetic_c64(int n, const float2* u, float2* out, const KinArgs& a, cudaStream_t stream);
int pairconv_c64_occupancy(int n, int mode, int blocks_per_sm);

// Batched launch over cells of unequal grid sides (batched.cu).
struct BatchCell {
  CUtensorMap tmap;     // the cell's partner array for the staged pipeline (sides with one)
  PairArgs pa;          // the cell's launch arguments (pa.out: final output or split buffer)
  float2* final_out;    // the cell's V_x u output
  int n;                // grid side
  int layout;           // staged sides: 0 LayoutOne, 1 LayoutSeq
};
struct BatchItem {
  int cell;             // index into the cell table
  int item;             // (split, k, tile) index within the cell
};
struct BatchArgs {
  const BatchCell* cells;
  const BatchItem* items;
  int nitems;
  int* counter;         // zeroed before each launch
  int* status;          // device status word
};
bool batched_side_supported(int n);
// Stage geometry of the side's staged pipeline in the batched launch (pitch and box rows of
// its tensor map); false for sides that run the pencil-load item there.
bool batched_stage_geometry(int n, int* sp, int* box_rows);
// Pencil layout of the 24^3 items of a batch: one pencil per thread (18 warps) or the ragged
// 12-warp form.
constexpr int kPencilOne = 0;
constexpr int kPencilRagged = 1;
// The persistent kernels of a batch: the pencil-load items, then the staged-partner items and
// the 12^3 LayoutOne items (any list may be empty).  With side, fork and join given, the staged
// kernels run on the side stream, forked from and joined back into `stream` (beside the pencil
// kernel; capturable), else after the pencil kernel on `stream`.
// pencil_blocked: every cell of the pencil-load list reads pencil-blocked copies (blk = 1).
cudaError_t launch_pairconv_batched(const BatchArgs& staged, const BatchArgs& staged12, const BatchArgs& pencil, int sms,
                                    int pencil_layout, bool pencil_blocked, cudaStream_t stream, cudaStream_t side,
                                    cudaEvent_t fork, cudaEvent_t join);

// One staged FP64 1-D transform pass along an axis of length L with element stride inner.
cudaError_t launch_staged_fft(int L, int dir, double2* work, size_t nbatch, int N, int inner, cudaStream_t stream);
bool staged_fft_supported(int L);

// Template body used by the per-size translation units.  `blocks_per_sm` selects the
// occupancy variant (1: registers uncapped; 2: two CTAs per SM where they fit).
template <int n, int MODE, int MINB, int PPT = 2, int TSX = Geo<n>::NN / PPT, bool TC = false, int BLK = -1>
cudaError_t pairconv_set_attr() {
  static bool attr_done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr_done[dev]) {
    cudaError_t err = cudaFuncSetAttribute(pairconv_c64_kernel<n, MODE, MINB, PPT, TSX, TC, BLK>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)pairconv_smem_request<n, TC>());
    if (err != cudaSuccess) return err;
    attr_done[dev] = true;
  }
  return cudaSuccess;
}

// BLK >= 0: the kernel compiled for that orbital layout (args.blk must match).
template <int n, int MODE, int MINB, int PPT, int TSX, bool TC, int BLK>
cudaError_t launch_pairconv_blk(const PairArgs& args, cudaStream_t stream) {
  cudaError_t err = pairconv_set_attr<n, MODE, MINB, PPT, TSX, TC, BLK>();
  if (err != cudaSuccess) return err;
  const dim3 grid(args.item_count > 0 ? (unsigned)args.item_count
                                      : (unsigned)((size_t)args.nsplit * args.nk_own * args.ntiles));
  pairconv_c64_kernel<n, MODE, MINB, PPT, TSX, TC, BLK>
      <<<grid, GeoP<n, PPT, TSX>::THREADS, pairconv_smem_request<n, TC>(), stream>>>(args);
  count_launch();
  return cudaGetLastError();
}

// One pencil per thread (the tightest register budget) has one kernel per orbital layout, so
// that the layout's address arithmetic is fixed at compile time; the other forms read it at
// run time.
template <int n, int MODE, int MINB, int PPT = 2, int TSX = Geo<n>::NN / PPT, bool TC = false>
cudaError_t launch_pairconv_variant(const PairArgs& args, cudaStream_t stream) {
  if constexpr (PPT == 1) {
    return args.blk ? launch_pairconv_blk<n, MODE, MINB, PPT, TSX, TC, 1>(args, stream)
                    : launch_pairconv_blk<n, MODE, MINB, PPT, TSX, TC, 0>(args, stream);
  } else {
    return launch_pairconv_blk<n, MODE, MINB, PPT, TSX, TC, -1>(args, stream);
  }
}

// Resident CTAs per SM of a variant (0 on error).
template <int n, int MODE, int MINB, int PPT = 2, int TSX = Geo<n>::NN / PPT, bool TC = false>
int pairconv_occupancy_variant() {
  constexpr int BLK = PPT == 1 ? 1 : -1;
  if (pairconv_set_attr<n, MODE, MINB, PPT, TSX, TC, BLK>() != cudaSuccess) return 0;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, pairconv_c64_kernel<n, MODE, MINB, PPT, TSX, TC, BLK>,
                                                    GeoP<n, PPT, TSX>::THREADS,
                                                    pairconv_smem_request<n, TC>()) != cudaSuccess)
    return 0;
  return blocks;
}

// Ragged pencil-load variant: 12 warps per owner slot (at most 3 on a warp scheduler, so up to
// 170 registers a thread); thread t takes pencil t and, for t < n^2 - 384, pencil t + 384.  For
// 24^3 (576 pencils) the busiest scheduler runs 5 pencil passes per stage instead of the 6 of
// two pencils per thread on 9 warps (3/2/2/2).
constexpr int kRaggedThreads = 384;
template <int n>
constexpr bool pencil_ragged_fits() {
  if constexpr (Geo<n>::T == 1 && Geo<n>::NN > kRaggedThreads && Geo<n>::NN <= 2 * kRaggedThreads &&
                (Geo<n>::NN - kRaggedThreads) % 32 == 0) {
    return GeoP<n, 2, kRaggedThreads>::TMEM_COLS <= 512;
  } else {
    return false;
  }
}

// Tensor-core variant (kTcVariant): the ragged pencil-load kernel with the Y and X stages as
// split-FP16 GEMMs (tc_dft.cuh), for the owner = target modes where 2n is a multiple of 16
// and the grids leave room for the DFT tables.
constexpr int kTcVariant = 4;
template <int n, int MODE>
constexpr bool tc_fits() {
  if constexpr (MODE != MODE_OCC && n % 8 == 0 && pencil_ragged_fits<n>()) {
    return Geo<n>::SMEM_BYTES + sizeof(TcTables<n>) <= 232448;
  } else {
    return false;
  }
}

// One-pencil variant (kOneVariant, the default where it fits): the pencil-load kernel with one
// pencil per thread, n^2 / 32 warps (24^3: 18 warps, 576 threads).  Every warp scheduler then
// holds 4-5 warps through a stage instead of 3 (the ragged form), at most 96 registers a thread
// (5 warps on the busiest scheduler's 16K-register file); its Z stages and folds move the
// orbitals and accumulators in small chunks to stay within them, and its orbital loads follow
// the L1 policy of pairconv_c64.cuh (kLdOwner, ...).  24^3, 4x4x4 k, 16 bands: 58.8 ms against
// 66.5 ms for the ragged form.  Owner = target modes only (the VJP's u_occ pass keeps the
// ragged form: its two chains and fused omega term need more registers).
constexpr int kOneVariant = 5;
template <int n>
constexpr bool pencil_one_fits() {
  if constexpr (Geo<n>::T == 1 && Geo<n>::NN % 32 == 0 && Geo<n>::NN <= 1024 && n % 4 == 0) {
    return GeoP<n, 1, Geo<n>::NN>::TMEM_COLS <= 512;
  } else {
    return false;
  }
}

// Staged-partner kernel (pairconv_tma.cuh): one CTA per SM.
// Encodes the tensor map of a partner array for the staged-partner kernel of side n.
cudaError_t make_partner_tmap(CUtensorMap* map, const void* base, int n, long long rows, int sp, int box_rows);

template <int n, int MODE, template <int> class L>
cudaError_t launch_pairconv_tma(const PairArgs& args, cudaStream_t stream) {
  using S = GeoS<n, L<n>>;
  static bool attr_done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr_done[dev]) {
    cudaError_t err = cudaFuncSetAttribute(pairconv_tma_kernel<n, MODE, L>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM_REQUEST);
    if (err != cudaSuccess) return err;
    attr_done[dev] = true;
  }
  CUtensorMap tmap;
  cudaError_t err = make_partner_tmap(&tmap, args.part, n, (long long)args.nk_part * args.n_part * Geo<n>::NN, S::SP, S::BR);
  if (err != cudaSuccess) return err;
  const dim3 grid((unsigned)((size_t)args.nsplit * args.nk_own * args.ntiles));
  pairconv_tma_kernel<n, MODE, L><<<grid, L<n>::THREADS, S::SMEM_REQUEST, stream>>>(args, tmap);
  count_launch();
  return cudaGetLastError();
}

// The staged-partner kernel exists for the owner = target modes and the layouts that fit.
template <int n, int MODE, template <int> class L>
constexpr bool tma_fits() {
  if constexpr (L<n>::OK && (MODE == MODE_APPLY || MODE == MODE_ENERGY || MODE == MODE_DOT)) {
    return GeoS<n, L<n>>::FITS;
  } else {
    return false;
  }
}

// Kernel variant: 0 the default (the staged-partner kernel with its default layout where it
// exists for (n, mode); else the one-pencil pencil-load kernel where it exists for (n, mode);
// else the ragged pencil-load kernel where it exists; else the pencil-load kernel at the
// occupancy the size allows); -1 / -2 the staged-partner kernel with LayoutSeq / LayoutOne;
// 1 or 2 the pencil-load kernel with that occupancy; 3 the ragged pencil-load kernel
// (pencil_ragged_fits; 24^3 99.6 -> 95.6 ms on the 4x4x4 k, 16-band cell against two pencils a
// thread on 9 warps); 4 (kTcVariant) its tensor-core form where tc_fits, else the ragged
// kernel; 5 (kOneVariant) the one-pencil pencil-load kernel where pencil_one_fits.
// A variant that does not exist for the size falls back to the default.
template <int n, int MODE>
constexpr int staged_layout(int variant) {
  if (variant > 0) return 0;
  const bool seq = tma_fits<n, MODE, LayoutSeq>(), one = tma_fits<n, MODE, LayoutOne>();
  if (variant == -1 && seq) return -1;
  if (variant == -2 && one) return -2;
  // default: one pencil per thread where it fits, else two
  return one ? -2 : (seq ? -1 : 0);
}

template <int n, int MODE>
cudaError_t launch_pairconv_mode(const PairArgs& args, int variant, cudaStream_t stream) {
  switch (staged_layout<n, MODE>(variant)) {
    case -1:
      if constexpr (tma_fits<n, MODE, LayoutSeq>()) return launch_pairconv_tma<n, MODE, LayoutSeq>(args, stream);
      break;
    case -2:
      if constexpr (tma_fits<n, MODE, LayoutOne>()) return launch_pairconv_tma<n, MODE, LayoutOne>(args, stream);
      break;
    default: break;
  }
  if constexpr (tc_fits<n, MODE>()) {
    if (variant == kTcVariant) return launch_pairconv_variant<n, MODE, 1, 2, kRaggedThreads, true>(args, stream);
  }
  if constexpr (pencil_one_fits<n>() && MODE != MODE_OCC) {
    if (variant == kOneVariant || variant <= 0)
      return launch_pairconv_variant<n, MODE, 1, 1, Geo<n>::NN>(args, stream);
  }
  if constexpr (pencil_ragged_fits<n>()) {
    if (variant >= 3 || variant <= 0) return launch_pairconv_variant<n, MODE, 1, 2, kRaggedThreads>(args, stream);
  }
  const int blocks_per_sm = (variant <= 0 || variant >= 3) ? 2 : variant;
  if (blocks_per_sm >= 2 && Geo<n>::MAXB >= 2) return launch_pairconv_variant<n, MODE, Geo<n>::MAXB>(args, stream);
  return launch_pairconv_variant<n, MODE, 1>(args, stream);
}

template <int n, int MODE>
int pairconv_occupancy_mode(int variant) {
  if (staged_layout<n, MODE>(variant) != 0) return 1;
  if constexpr (tc_fits<n, MODE>()) {
    if (variant == kTcVariant) return pairconv_occupancy_variant<n, MODE, 1, 2, kRaggedThreads, true>();
  }
  if constexpr (pencil_one_fits<n>() && MODE != MODE_OCC) {
    if (variant == kOneVariant || variant <= 0) return pairconv_occupancy_variant<n, MODE, 1, 1, Geo<n>::NN>();
  }
  if constexpr (pencil_ragged_fits<n>()) {
    if (variant >= 3 || variant <= 0) return pairconv_occupancy_variant<n, MODE, 1, 2, kRaggedThreads>();
  }
  const int blocks_per_sm = (variant <= 0 || variant >= 3) ? 2 : variant;
  if (blocks_per_sm >= 2 && Geo<n>::MAXB >= 2) return pairconv_occupancy_variant<n, MODE, Geo<n>::MAXB>();
  return pairconv_occupancy_variant<n, MODE, 1>();
}

// Whether (n, mode, variant) runs the pencil-load kernel (which reads the pencil-blocked
// orbital layout when PairArgs::blk is set) rather than the staged-partner one.
template <int n>
bool pencil_load_n(int mode, int variant) {
  switch (mode) {
    case MODE_APPLY: return staged_layout<n, MODE_APPLY>(variant) == 0;
    case MODE_ENERGY: return staged_layout<n, MODE_ENERGY>(variant) == 0;
    case MODE_DOT: return staged_layout<n, MODE_DOT>(variant) == 0;
    default: return true;
  }
}

template <int n>
cudaError_t launch_pairconv_c64_n(int mode, const PairArgs& args, int blocks_per_sm, cudaStream_t stream) {
  switch (mode) {
    case MODE_APPLY: return launch_pairconv_mode<n, MODE_APPLY>(args, blocks_per_sm, stream);
    case MODE_ENERGY: return launch_pairconv_mode<n, MODE_ENERGY>(args, blocks_per_sm, stream);
    case MODE_DOT: return launch_pairconv_mode<n, MODE_DOT>(args, blocks_per_sm, stream);
    case MODE_OCC: return launch_pairconv_mode<n, MODE_OCC>(args, blocks_per_sm, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <int n>
int pairconv_occupancy_n(int mode, int blocks_per_sm) {
  switch (mode) {
    case MODE_APPLY: return pairconv_occupancy_mode<n, MODE_APPLY>(blocks_per_sm);
    case MODE_ENERGY: return pairconv_occupancy_mode<n, MODE_ENERGY>(blocks_per_sm);
    case MODE_DOT: return pairconv_occupancy_mode<n, MODE_DOT>(blocks_per_sm);
    case MODE_OCC: return pairconv_occupancy_mode<n, MODE_OCC>(blocks_per_sm);
    default: return 0;
  }
}

}  // namespace hse
