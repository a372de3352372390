// pairconv_tma.cuh - fused FP32 pair-convolution kernel with the partner orbital staged by TMA
// and the owner orbital resident in Tensor Memory.
//
// Same chain as pairconv_c64.cuh (Sec. II C, Eq. "Fock" / "Fock-DS": pair density, 3-D FFT,
// kernel multiply, inverse FFT, multiply-accumulate), reorganised so that the orbitals cross
// the L2 -> SM path once:
//   * the owner orbital(s) u_i are copied into TMEM once per CTA (beside the accumulators and
//     the per-k' kernel rows);
//   * each partner u_j is brought into shared memory by 2-D tensor copies (TMA): the orbital
//     is viewed as rows of one z-pencil (2n floats) and each box row lands at a padded pitch SP
//     (the box is wider than the pencil, the excess is out-of-bounds and zero-filled), so the
//     128-bit reads of the Z stages are free of bank conflicts; double-buffered: the copy for
//     the next pair is issued right after the first barrier of the current pair and completes
//     on an mbarrier while the current pair is in its Y, X and inverse stages;
//   * every mbarrier wait is bounded in time; on expiry the kernel records HSE_ERR_TIMEOUT in
//     the status word, stops issuing copies and finishes without waiting further.
// One CTA per SM (it takes all 512 TMEM columns); the T owner slots of a CTA share each
// staged partner.
#pragma once

#include <cuda.h>

#include "pairconv_c64.cuh"
#include "tma.cuh"

namespace hse {

constexpr int kStatusTimeout = -5;  // HSE_ERR_TIMEOUT
constexpr int kStatusDevice = -7;   // HSE_ERR_DEVICE

// Stage buffer of one partner orbital: NB tensor boxes of BR z-pencils at pitch SP.
template <int n>
struct StageGeo {
  using G = Geo<n>;
  static constexpr int SP = ((n / 2) % 2 == 1) ? n : n + 2;    // stage pencil pitch (complex)
  static constexpr int NB = (G::NN + 255) / 256;                // tensor boxes per fill
  static constexpr int BR = (((G::NN + NB - 1) / NB) + 7) / 8 * 8;  // rows (pencils) per box
  static constexpr int STAGE_ROWS = NB * BR;
  static constexpr int STAGE_CPX = STAGE_ROWS * SP;             // one stage buffer
  static constexpr int STAGE_TX = STAGE_ROWS * SP * 8;          // bytes one fill delivers
};

// Shared and tensor memory of the staged kernel for pencil layout Lay (below).
template <int n, class Lay>
struct GeoS : StageGeo<n> {
  using G = Geo<n>;
  using SG = StageGeo<n>;
  static constexpr size_t GRIDS_BYTES = ((size_t)G::T * Lay::GRID_CPX * sizeof(float2) + 127) / 128 * 128;
  static constexpr int COLS_PER_WARP = Lay::COLS_PER_WARP;
  static constexpr int TMEM_COLS = pow2_at_least(((Lay::WARPS + 3) / 4) * COLS_PER_WARP);
  static constexpr size_t SMEM_BYTES = GRIDS_BYTES + 2 * (size_t)SG::STAGE_CPX * sizeof(float2);
  // + 128 bytes to align the base at run time; at least enough that a second CTA (which would
  // need TMEM too) never fits
  static constexpr size_t SMEM_REQUEST = SMEM_BYTES + 128 > 118784 ? SMEM_BYTES + 128 : 118784;
  // 4.5 KB of static shared memory (occupation cache, barriers) sit beside the dynamic part
  static constexpr bool FITS =
      Lay::OK && TMEM_COLS <= 512 && SMEM_REQUEST + 4608 <= 232448 && Lay::THREADS <= 1024;
};

// Z forward for the PPT pencils: rho = conj(u_j) u_i with u_j from the stage, u_i from TMEM.
template <int n, int PPT>
__device__ __forceinline__ void stage_z_forward_staged(float2* g, int t, bool valid, const float2* stg, uint32_t town) {
  using G = Geo<n>;
  using S = StageGeo<n>;
#pragma unroll 1
  for (int ps = 0; ps < PPT; ++ps) {
    const Pencil<n> pc(t + ps * (G::NN / PPT));
    float uo[G::ROW];
    TmemRow<G::ROW>::load(town + (uint32_t)(ps * G::ROW), uo);
    const float4* s4 = reinterpret_cast<const float4*>(stg + (pc.zg / n) * S::SP);
    cpx<float> v[n];
#pragma unroll
    for (int e = 0; e < n / 2; ++e) {
      const float4 w = s4[e];  // u_j at z = 2e, 2e+1
      v[2 * e] = {w.x * uo[4 * e] + w.y * uo[4 * e + 1], w.x * uo[4 * e + 1] - w.y * uo[4 * e]};
      v[2 * e + 1] = {w.z * uo[4 * e + 2] + w.w * uo[4 * e + 3], w.z * uo[4 * e + 3] - w.w * uo[4 * e + 2]};
    }
    fft<n, -1, float>(v);
    if (valid) store_s<n, G::ZVEC>(v, g, pc.zs, 1);
  }
}

// Z inverse for the PPT pencils, acc += u_j phi with u_j from the stage.  Warp-wide (TMEM).
template <int n, int PPT>
__device__ __forceinline__ void stage_z_inverse_staged(const float2* g, int t, const float2* stg, uint32_t trow0) {
  using G = Geo<n>;
  using S = StageGeo<n>;
#pragma unroll 1
  for (int ps = 0; ps < PPT; ++ps) {
    const Pencil<n> pc(t + ps * (G::NN / PPT));
    cpx<float> v[n];
    load_s<n, G::ZVEC>(v, g, pc.zs, 1);
    fft<n, +1, float>(v);
    float acc[G::ROW];
    const uint32_t trow = trow0 + (uint32_t)(ps * G::ROW);
    TmemRow<G::ROW>::load(trow, acc);
    const float4* s4 = reinterpret_cast<const float4*>(stg + (pc.zg / n) * S::SP);
#pragma unroll
    for (int e = 0; e < n / 2; ++e) {
      const float4 w = s4[e];
      float* a = acc + 4 * e;
      a[0] = fmaf(w.x, v[2 * e].x, fmaf(-w.y, v[2 * e].y, a[0]));
      a[1] = fmaf(w.x, v[2 * e].y, fmaf(w.y, v[2 * e].x, a[1]));
      a[2] = fmaf(w.z, v[2 * e + 1].x, fmaf(-w.w, v[2 * e + 1].y, a[2]));
      a[3] = fmaf(w.z, v[2 * e + 1].y, fmaf(w.w, v[2 * e + 1].x, a[3]));
    }
    TmemRow<G::ROW>::store(trow, acc);
  }
}

// ---------------------------------------------------------------------------------------
// Pencil layouts of the staged kernel.  A layout says how many pencils each thread owns per
// stage (PPT), hence the block size, which pencils they are, and where its TMEM columns sit
// (relative to the warp's first column trow0); the pipeline is the same.
//   LayoutSeq:   two pencils per thread (t and t + n^2/2), transformed one after the other.
//   LayoutOne:   one pencil per thread, twice the warps.  The n^2 pencils of a stage are spread
//                over the four warp schedulers of the SM; one pencil per thread leaves the
//                busiest scheduler fewer pencil passes when n^2 / 128 has a small fractional
//                part (18^3: 3 instead of 4) and gives each scheduler more warps to hide
//                shared-memory latency.  Its X stage takes the pencils in the bank-spread
//                order of x_pencil (no bank conflicts where the pitch P differs from n).
// TMEM columns of a warp: [acc (PPT pencils) | kernel rows (PPT) | owner u_i (PPT) |
// running sums s, c (PPT, where they fit)].
// ---------------------------------------------------------------------------------------

// XP: with one pencil per thread, the X-stage pencils go to threads in the bank-spread order
// of x_pencil.
template <int n, int PPT_, bool XP = (PPT_ == 1)>
struct LayoutLin {
  using G = Geo<n>;
  static constexpr int PPT = PPT_;
  static constexpr int TS = G::NN / PPT;                          // threads per owner slot
  static constexpr int THREADS = (G::T * TS + 31) / 32 * 32;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int GRID_CPX = G::GRID_CPX;
  static constexpr bool OK = G::ZFAST_Y == 1 && THREADS <= 1024;
  static constexpr int TAB = PPT * G::ROW;
  static constexpr int OWN = TAB + PPT * n;
  // Where the lane quarters have room (the warps sharing one quarter take at most 512
  // columns), the running sums of the compensated accumulation live in TMEM too: s (ROW
  // floats) at SUMS + ps ROW and c (n columns of bf16 pairs) at CSUM + ps n.  Elsewhere
  // (20^3: four warps share a quarter) they live in global memory (PairArgs::comp).
  static constexpr int BASE = OWN + PPT * G::ROW;
  static constexpr int SUMCOLS = PPT * (G::ROW + n);
  static constexpr bool TSUMS = ((THREADS / 32 + 3) / 4) * (BASE + SUMCOLS) <= 512;
  static constexpr int SUMS = BASE;
  static constexpr int CSUM = BASE + PPT * G::ROW;
  static constexpr int COLS_PER_WARP = BASE + (TSUMS ? SUMCOLS : 0);
  static __device__ __forceinline__ int zg(int t, int ps) { return Pencil<n>(t + ps * TS).zg; }
  static __device__ __forceinline__ void z_forward(float2* g, int t, bool valid, const float2* stg, uint32_t trow0) {
    stage_z_forward_staged<n, PPT>(g, t, valid, stg, trow0 + (uint32_t)OWN);
  }
  static __device__ __forceinline__ void z_inverse(const float2* g, int t, const float2* stg, uint32_t trow0) {
    stage_z_inverse_staged<n, PPT>(g, t, stg, trow0);
  }
  template <int DIR>
  static __device__ __forceinline__ void y(float2* g, int t, bool valid) {
    stage_y<n, DIR, PPT>(g, t, valid);
  }
  static __device__ __forceinline__ void x(float2* g, int t, bool valid, uint32_t trow0, float f) {
    stage_x<n, PPT, XP>(g, t, valid, trow0 + (uint32_t)TAB, f);
  }
  static __device__ __forceinline__ void cache_row(int t, uint32_t trow0, const float* vrow, float scale) {
    cache_kernel_row<n, PPT, XP>(t, trow0 + (uint32_t)TAB, vrow, scale);
  }
  // Warp-local planes.  Pencil p of the Z and Y stages lies in the x-plane p / n; when n
  // divides 32, the 32 consecutive pencils of a warp's pass are 32 / n whole planes in both
  // stages (and a warp never straddles two owner slots), so the Y stage after a Z stage and the
  // Z stage after a Y stage read only what the same warp wrote: __syncwarp replaces the block
  // barrier there, and only the X stage, which reads every plane, keeps block barriers.  (Groups
  // of several warps under named barriers measured slower: 20^3 34.6 -> 35.9 ms, 18^3 1.23 ->
  // 1.25 ms; warp-local 16^3 14.40 -> 14.23 ms, 8^3 1.87 -> 1.84 ms.)
  static constexpr bool GROUPED = 32 % n == 0 && (G::T == 1 || TS % 32 == 0);
  static __device__ __forceinline__ void group_sync(int) { __syncwarp(); }
};

template <int n>
struct LayoutSeq : LayoutLin<n, 2> {};
template <int n>
struct LayoutOne : LayoutLin<n, 1> {};

// Occupations of one work item's partners, cached in shared memory when they fit.
constexpr int kOccCache = 1024;

// Occupation of partner q of the item (q = (kp - kp_begin) * n_part + j): from the shared
// cache, or from global memory past its end.
__device__ __forceinline__ float item_occ(const float* occ_sh, const PairArgs& a, int kp_begin, int q) {
  if (q < kOccCache) return occ_sh[q];
  const int kp = kp_begin + q / a.n_part, j = q - (q / a.n_part) * a.n_part;
  return (float)a.occ[kp * a.n_occ + j];
}

// Next partner index q' >= q with nonzero occupation.
__device__ __forceinline__ int next_partner(const float* occ_sh, const PairArgs& a, int kp_begin, int q, int npairs) {
  while (q < npairs && item_occ(occ_sh, a, kp_begin, q) == 0.f) ++q;
  return q;
}

// Pipeline state of the staged kernel that lives in shared memory beside the grids and
// persists across the work items of a persistent launch.
struct StagedShared {
  uint64_t mbar[2];   // stage buffer b's copy has landed
  int abort;          // a bounded wait expired: issue and wait no more
  float occ[kOccCache];
};

// One work item (split, k, owner tile) of the staged-partner pipeline: the item's partners
// stream through the two stage buffers, the owner orbital and the accumulators stay in TMEM.
// tmap: the partner array as rows of z-pencils, box {2 SP floats, BR rows} (in kernel
// parameter space or global memory).  phase0 / phase1: the parities the stage barriers are
// expected to complete next (carried from item to item).  on: this thread's warp takes part
// (a persistent block may be larger than the layout's); every thread of the block must call
// this, because it synchronises the block.  sbase must be 128-byte aligned.  Returns false
// after a timed-out wait (the caller stops).
template <int n, int MODE, template <int> class L>
__device__ __forceinline__ bool staged_item(const PairArgs& args, const CUtensorMap* tmap, int item, char* sbase,
                                            uint32_t tbase, StagedShared& sh, uint32_t& phase0, uint32_t& phase1,
                                            bool on) {
  using G = Geo<n>;
  using Lay = L<n>;
  using S = GeoS<n, Lay>;
  static_assert(MODE == MODE_APPLY || MODE == MODE_ENERGY || MODE == MODE_DOT, "owner = target modes only");
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const bool valid = on && tid < G::T * Lay::TS;
  const int slot = valid ? tid / Lay::TS : 0;
  const int t = valid ? tid - slot * Lay::TS : 0;
  float2* grids = reinterpret_cast<float2*>(sbase);
  float2* g = grids + slot * Lay::GRID_CPX;
  float2* stage = reinterpret_cast<float2*>(sbase + S::GRIDS_BYTES);
  const uint32_t trow0 = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * S::COLS_PER_WARP);
  const uint32_t town = trow0 + (uint32_t)Lay::OWN;

  const ItemIdx it(args, item);
  const int split = it.split;
  const int k = it.k;
  const int band = it.tile * G::T + slot;
  const bool active = valid && band < args.n_own;
  const int bandc = active ? band : 0;
  const int kp_begin = (int)(((long long)split * args.nk_part) / args.nsplit);
  const int kp_end = (int)(((long long)(split + 1) * args.nk_part) / args.nsplit);
  const int npairs = (kp_end - kp_begin) * args.n_part;
  const float2* own = args.own + ((size_t)k * args.n_own + bandc) * G::N;

  // fill stage buffer `buf` with partner q (warp 0 only)
  auto fill = [&](int q, int buf) {
    if (lane == 0) {
      const int kp = kp_begin + q / args.n_part, j = q - (q / args.n_part) * args.n_part;
      const int row0 = (kp * args.n_part + j) * G::NN;
      float2* dst = stage + buf * S::STAGE_CPX;
      mbar_arrive_expect_tx(&sh.mbar[buf], (uint32_t)S::STAGE_TX);
#pragma unroll
      for (int b = 0; b < S::NB; ++b) tensor_copy_2d_g2s(dst + b * S::BR * S::SP, tmap, 0, row0 + b * S::BR, &sh.mbar[buf]);
    }
    __syncwarp();
  };

  // the item's partner occupations, once (work items are sized so that they fit)
  for (int i = tid; i < npairs && i < kOccCache; i += blockDim.x) {
    const int kp = kp_begin + i / args.n_part, j = i - (i / args.n_part) * args.n_part;
    sh.occ[i] = (float)args.occ[kp * args.n_occ + j];
  }
  __syncthreads();
  int q = next_partner(sh.occ, args, kp_begin, 0, npairs);
  if (warp == 0 && q < npairs && args.inject != 1 && !sh.abort) {
    fence_proxy_async_smem();  // earlier generic accesses to this shared memory come first
    fill(q, 0);
  }

  // owner orbital into TMEM, accumulators to zero
  const bool reg = on;  // warp-uniform
#pragma unroll 1
  for (int ps = 0; ps < (reg ? Lay::PPT : 0); ++ps) {
    cpx<float> w[n];
    load_pencil_global<n>(w, own + Lay::zg(t, ps));
    float r[G::ROW];
#pragma unroll
    for (int e = 0; e < n; ++e) {
      r[2 * e] = w[e].x;
      r[2 * e + 1] = w[e].y;
    }
    TmemRow<G::ROW>::store(town + (uint32_t)(ps * G::ROW), r);
#pragma unroll
    for (int e = 0; e < G::ROW; ++e) r[e] = 0.f;
    TmemRow<G::ROW>::store(trow0 + (uint32_t)(ps * G::ROW), r);
  }

  // compensated accumulation over the k' groups of the item: APPLY keeps the running sums in
  // its output region (s) and in args.comp (c); ENERGY / DOT add group dots to dsum (FP64)
  const size_t oofs = split * args.split_stride + ((size_t)k * args.n_own + bandc) * G::N;
  float4* sums = (MODE == MODE_APPLY) ? sums_of(args, oofs / G::N, OrbBlk<n>::NBK) : nullptr;
  const float2* lhs = (MODE == MODE_DOT) ? args.part2 + ((size_t)k * args.n_own + bandc) * G::N : own;
  double dsum = 0.0;
  int folds = 0;
  const int fspan = fold_span(args.n_part);
  auto fold = [&](bool last) {
#pragma unroll 1
    for (int ps = 0; ps < (reg ? Lay::PPT : 0); ++ps) {
      const uint32_t trow = trow0 + (uint32_t)(ps * G::ROW);
      float acc[G::ROW];
      TmemRow<G::ROW>::load(trow, acc);
      if constexpr (MODE == MODE_APPLY && Lay::TSUMS) {
        const int zg = Lay::zg(t, ps);
        fold_group_tmem<n>(acc, trow0 + (uint32_t)(Lay::SUMS + ps * G::ROW), trow0 + (uint32_t)(Lay::CSUM + ps * n),
                           active ? reinterpret_cast<float4*>(args.out + oofs + zg) : nullptr, folds == 0,
                           folds == 1, last);
      } else if constexpr (MODE == MODE_APPLY) {
        if (active) {
          const int zg = Lay::zg(t, ps);
          fold_group<n>(acc, sums, zg / n, reinterpret_cast<float4*>(args.out + oofs + zg), folds == 0, folds == 1,
                        last);
        }
      } else {
        cpx<float> w[n];
        if constexpr (MODE == MODE_ENERGY) {
          float r[G::ROW];
          TmemRow<G::ROW>::load(town + (uint32_t)(ps * G::ROW), r);
#pragma unroll
          for (int e = 0; e < n; ++e) w[e] = {r[2 * e], r[2 * e + 1]};
        } else {
          load_pencil_global<n>(w, lhs + Lay::zg(t, ps));
        }
        dsum += (double)pencil_dot<n>(w, acc);
      }
      if (!last) {
#pragma unroll
        for (int e = 0; e < G::ROW; ++e) acc[e] = 0.f;
        TmemRow<G::ROW>::store(trow, acc);
      }
    }
    ++folds;
  };

  int buf = 0;
  int cur_kp = -1;
  while (q < npairs) {
    const int kp = kp_begin + q / args.n_part;
    const float f = item_occ(sh.occ, args, kp_begin, q);
    if (kp != cur_kp) {
      // a new fold group (fold_span k-points) starts: fold the previous one
      if (cur_kp >= 0 && (kp - kp_begin) / fspan != (cur_kp - kp_begin) / fspan) fold(false);
      const int qrow = args.qidx[k * args.nk_part + kp];
      if (on) Lay::cache_row(t, trow0, args.vtab + (size_t)qrow * G::N, args.scale);
      cur_kp = kp;
    }
    // partner u_j has landed in stage[buf]
    const uint32_t ph = buf ? phase1 : phase0;
    if (!sh.abort) {
      if (!mbar_wait_bounded(&sh.mbar[buf], ph)) {
        sh.abort = 1;
        if (args.status) atomicExch(args.status, kStatusTimeout);
      }
    }
    if (buf) phase1 ^= 1u; else phase0 ^= 1u;
    const float2* stg = stage + buf * S::STAGE_CPX;
    const int qn = next_partner(sh.occ, args, kp_begin, q + 1, npairs);
    // refill stage[buf ^ 1] with the next partner once every thread is past its last read of it
    // (the previous pair's Z inverse)
    auto refill = [&]() {
      if (warp == 0 && qn < npairs && !sh.abort) {
        fence_proxy_async_smem();
        fill(qn, buf ^ 1);
      }
    };
    if (on) Lay::z_forward(g, t, valid, stg, trow0);
    if constexpr (Lay::GROUPED) {
      if (on) Lay::group_sync(tid);
    } else {
      __syncthreads();
      refill();
    }
    if (on) Lay::template y<-1>(g, t, valid);
    __syncthreads();
    if constexpr (Lay::GROUPED) refill();
    if (on) Lay::x(g, t, valid, trow0, f);
    __syncthreads();
    if (on) Lay::template y<+1>(g, t, valid);
    if constexpr (Lay::GROUPED) {
      if (on) Lay::group_sync(tid);
    } else {
      __syncthreads();
    }
    if (on) Lay::z_inverse(g, t, stg, trow0);
    q = qn;
    buf ^= 1;
  }
  __syncthreads();
  const bool ok = !sh.abort;
  if (!ok && tid == 0) {
    // a copy may still be in flight after a timeout: give it one more bounded chance to land
    mbar_wait_bounded(&sh.mbar[0], phase0);
    mbar_wait_bounded(&sh.mbar[1], phase1);
  }

  // the last group (with no partner at all, the accumulators still hold zeros: one fold
  // writes them)
  fold(true);
  if constexpr (MODE != MODE_APPLY) {
    const double d = dsum;
    __syncthreads();
    double* red = reinterpret_cast<double*>(sbase);
    red[tid] = valid ? d : 0.0;
    __syncthreads();
    if (valid && t == 0 && active) {
      double sum = 0.0;
      for (int e = 0; e < Lay::TS; ++e) sum += red[slot * Lay::TS + e];
      if (MODE == MODE_ENERGY) sum *= args.occ_own[k * args.n_occ + band];
      args.partial[split * args.split_stride + (size_t)k * args.n_own + band] = sum;
    }
  }
  __syncthreads();  // the grids, the reduction scratch and the occupation cache are reused next
  return ok;
}

// Aligns the dynamic shared memory base to 128 bytes for TMA (128 bytes of slack are
// requested); null (and the status word set) should it still not be aligned.
__device__ __forceinline__ char* staged_smem_base(float4* smem4, int* status) {
  char* sbase = reinterpret_cast<char*>(smem4);
  sbase += (128u - (smem_addr_u32(sbase) & 127u)) & 127u;
  if ((smem_addr_u32(sbase) & 127u) != 0) {
    if (threadIdx.x == 0 && status) atomicExch(status, kStatusDevice);
    return nullptr;
  }
  return sbase;
}

// One work item per CTA.  L: the pencil layout (LayoutSeq or LayoutOne).
template <int n, int MODE, template <int> class L>
__global__ void __launch_bounds__(L<n>::THREADS, 1)
    pairconv_tma_kernel(const PairArgs args, const __grid_constant__ CUtensorMap tmap) {
  using S = GeoS<n, L<n>>;
  extern __shared__ __align__(128) float4 smem4[];
  __shared__ uint32_t tmem_base_sh;
  __shared__ StagedShared sh;
  char* sbase = staged_smem_base(smem4, args.status);
  if (!sbase) return;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(&sh.mbar[0], 1);
    mbar_init(&sh.mbar[1], 1);
    sh.abort = 0;
    mbar_fence_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base_sh, S::TMEM_COLS);
    tmem_relinquish();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  uint32_t phase0 = 0, phase1 = 0;
  staged_item<n, MODE, L>(args, &tmap, blockIdx.x, sbase, tmem_base_sh, sh, phase0, phase1, true);
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem_base_sh, S::TMEM_COLS);
}

}  // namespace hse
