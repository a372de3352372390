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

template <int n>
struct GeoS {
  using G = Geo<n>;
  static constexpr int SP = ((n / 2) % 2 == 1) ? n : n + 2;    // stage pencil pitch (complex)
  static constexpr int NB = (G::NN + 255) / 256;                // tensor boxes per fill
  static constexpr int BR = (((G::NN + NB - 1) / NB) + 7) / 8 * 8;  // rows (pencils) per box
  static constexpr int STAGE_ROWS = NB * BR;
  static constexpr int STAGE_CPX = STAGE_ROWS * SP;             // one stage buffer
  static constexpr int STAGE_TX = STAGE_ROWS * SP * 8;          // bytes one fill delivers
  static constexpr size_t GRIDS_BYTES = ((size_t)G::T * G::GRID_CPX * sizeof(float2) + 127) / 128 * 128;
  static constexpr int TAB = 2 * G::ROW;                        // [acc0 acc1 | tab0 tab1 | own0 own1]
  static constexpr int OWN = TAB + 2 * n;
  static constexpr int COLS_PER_WARP = OWN + 2 * G::ROW;
  static constexpr int TMEM_COLS = pow2_at_least(((G::WARPS + 3) / 4) * COLS_PER_WARP);
  static constexpr size_t SMEM_BYTES = GRIDS_BYTES + 2 * (size_t)STAGE_CPX * sizeof(float2);
  // + 128 bytes to align the base at run time; at least enough that a second CTA (which would
  // need TMEM too) never fits
  static constexpr size_t SMEM_REQUEST = SMEM_BYTES + 128 > 118784 ? SMEM_BYTES + 128 : 118784;
  static constexpr bool FITS = TMEM_COLS <= 512 && SMEM_REQUEST + 1024 <= 232448 && G::ZFAST_Y == 1;
};

// Z forward for both pencils: rho = conj(u_j) u_i with u_j from the stage and u_i from TMEM.
template <int n>
__device__ __forceinline__ void stage_z_forward_staged(float2* g, int t, bool valid, const float2* stg, uint32_t town) {
  using G = Geo<n>;
  using S = GeoS<n>;
#pragma unroll 1
  for (int ps = 0; ps < 2; ++ps) {
    const Pencil<n> pc(t + ps * G::TS);
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

// Z inverse for both pencils, acc += u_j phi with u_j from the stage.  Warp-wide (TMEM).
template <int n>
__device__ __forceinline__ void stage_z_inverse_staged(const float2* g, int t, const float2* stg, uint32_t trow0) {
  using G = Geo<n>;
  using S = GeoS<n>;
#pragma unroll 1
  for (int ps = 0; ps < 2; ++ps) {
    const Pencil<n> pc(t + ps * G::TS);
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

// tmap: the partner array as rows of z-pencils, box {2 SP floats, BR rows}.
template <int n, int MODE>
__global__ void __launch_bounds__(Geo<n>::THREADS, 1)
    pairconv_tma_kernel(const PairArgs args, const __grid_constant__ CUtensorMap tmap) {
  using G = Geo<n>;
  using S = GeoS<n>;
  static_assert(MODE == MODE_APPLY || MODE == MODE_ENERGY || MODE == MODE_DOT, "owner = target modes only");
  extern __shared__ __align__(128) float4 smem4[];
  __shared__ uint32_t tmem_base_sh;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ int abort_sh;
  __shared__ float occ_sh[kOccCache];

  const int tid = threadIdx.x;
  // TMA destinations must be 128-byte aligned: align the dynamic shared memory base (128 bytes
  // of slack are requested), and refuse to run, recording the failure, should it still not be.
  char* sbase = reinterpret_cast<char*>(smem4);
  sbase += (128u - (smem_addr_u32(sbase) & 127u)) & 127u;
  if ((smem_addr_u32(sbase) & 127u) != 0) {
    if (tid == 0 && args.status) atomicExch(args.status, kStatusDevice);
    return;
  }
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const bool valid = tid < G::T * G::TS;
  const int slot = valid ? tid / G::TS : 0;
  const int t = valid ? tid - slot * G::TS : 0;
  float2* grids = reinterpret_cast<float2*>(sbase);
  float2* g = grids + slot * G::GRID_CPX;
  float2* stage = reinterpret_cast<float2*>(sbase + S::GRIDS_BYTES);

  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    abort_sh = 0;
    mbar_fence_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base_sh, S::TMEM_COLS);
    tmem_relinquish();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tbase = tmem_base_sh;
  const uint32_t trow0 = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * S::COLS_PER_WARP);
  const uint32_t ttab = trow0 + (uint32_t)S::TAB;
  const uint32_t town = trow0 + (uint32_t)S::OWN;

  const int per_split = args.nk * args.ntiles;
  const int split = blockIdx.x / per_split;
  const int rem = blockIdx.x - split * per_split;
  const int k = rem / args.ntiles;
  const int band = (rem - k * args.ntiles) * G::T + slot;
  const bool active = valid && band < args.n_own;
  const int bandc = active ? band : 0;
  const int kp_begin = (int)(((long long)split * args.nk) / args.nsplit);
  const int kp_end = (int)(((long long)(split + 1) * args.nk) / args.nsplit);
  const int npairs = (kp_end - kp_begin) * args.n_part;
  const float2* own = args.own + ((size_t)k * args.n_own + bandc) * G::N;

  // fill stage buffer `buf` with partner q (warp 0 only)
  auto fill = [&](int q, int buf) {
    if (lane == 0) {
      const int kp = kp_begin + q / args.n_part, j = q - (q / args.n_part) * args.n_part;
      const int row0 = (kp * args.n_part + j) * G::NN;
      float2* dst = stage + buf * S::STAGE_CPX;
      mbar_arrive_expect_tx(&mbar[buf], (uint32_t)S::STAGE_TX);
#pragma unroll
      for (int b = 0; b < S::NB; ++b) tensor_copy_2d_g2s(dst + b * S::BR * S::SP, &tmap, 0, row0 + b * S::BR, &mbar[buf]);
    }
    __syncwarp();
  };

  // the item's partner occupations, once (work items are sized so that they fit)
  for (int i = tid; i < npairs && i < kOccCache; i += blockDim.x) {
    const int kp = kp_begin + i / args.n_part, j = i - (i / args.n_part) * args.n_part;
    occ_sh[i] = (float)args.occ[kp * args.n_occ + j];
  }
  __syncthreads();
  int q = next_partner(occ_sh, args, kp_begin, 0, npairs);
  if (warp == 0 && q < npairs && args.inject != 1) fill(q, 0);

  // owner orbital into TMEM, accumulators to zero
#pragma unroll 1
  for (int ps = 0; ps < 2; ++ps) {
    const Pencil<n> pc(t + ps * G::TS);
    cpx<float> w[n];
    load_pencil_global<n>(w, own + pc.zg);
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

  uint32_t phase0 = 0, phase1 = 0;
  int buf = 0;
  int cur_kp = -1;
  while (q < npairs) {
    const int kp = kp_begin + q / args.n_part;
    const float f = item_occ(occ_sh, args, kp_begin, q);
    if (kp != cur_kp) {
      const int qrow = args.qidx[k * args.nk + kp];
      cache_kernel_row<n>(t, ttab, args.vtab + (size_t)qrow * G::N, args.scale);
      cur_kp = kp;
    }
    // partner u_j has landed in stage[buf]
    const uint32_t ph = buf ? phase1 : phase0;
    if (!abort_sh) {
      if (!mbar_wait_bounded(&mbar[buf], ph)) {
        abort_sh = 1;
        if (args.status) atomicExch(args.status, kStatusTimeout);
      }
    }
    if (buf) phase1 ^= 1u; else phase0 ^= 1u;
    const float2* stg = stage + buf * S::STAGE_CPX;
    stage_z_forward_staged<n>(g, t, valid, stg, town);
    __syncthreads();
    // every thread is past its last read of stage[buf ^ 1]: refill it with the next partner
    const int qn = next_partner(occ_sh, args, kp_begin, q + 1, npairs);
    if (warp == 0 && qn < npairs && !abort_sh) {
      fence_proxy_async_smem();
      fill(qn, buf ^ 1);
    }
    stage_y<n, -1>(g, t, valid);
    __syncthreads();
    stage_x<n>(g, t, valid, ttab, f);
    __syncthreads();
    stage_y<n, +1>(g, t, valid);
    __syncthreads();
    stage_z_inverse_staged<n>(g, t, stg, trow0);
    q = qn;
    buf ^= 1;
  }
  __syncthreads();
  if (abort_sh && tid == 0) {
    // a copy may still be in flight after a timeout: give it one more bounded chance to land
    mbar_wait_bounded(&mbar[0], phase0);
    mbar_wait_bounded(&mbar[1], phase1);
  }

  if constexpr (MODE == MODE_APPLY) {
    float2* obase = args.out + split * args.split_stride + ((size_t)k * args.n_own + bandc) * G::N;
#pragma unroll 1
    for (int ps = 0; ps < 2; ++ps) {
      const Pencil<n> pc(t + ps * G::TS);
      float acc[G::ROW];
      TmemRow<G::ROW>::load(trow0 + (uint32_t)(ps * G::ROW), acc);
      if (active) {
        float4* o = reinterpret_cast<float4*>(obase + pc.zg);
#pragma unroll
        for (int e = 0; e < n / 2; ++e) o[e] = make_float4(acc[4 * e], acc[4 * e + 1], acc[4 * e + 2], acc[4 * e + 3]);
      }
    }
  } else {
    const float2* lhs = (MODE == MODE_ENERGY) ? own : args.part2 + ((size_t)k * args.n_own + bandc) * G::N;
    double d = 0.0;
#pragma unroll 1
    for (int ps = 0; ps < 2; ++ps) {
      const Pencil<n> pc(t + ps * G::TS);
      float acc[G::ROW];
      TmemRow<G::ROW>::load(trow0 + (uint32_t)(ps * G::ROW), acc);
      cpx<float> w[n];
      load_pencil_global<n>(w, lhs + pc.zg);
#pragma unroll
      for (int e = 0; e < n; ++e) d += (double)w[e].x * (double)acc[2 * e] + (double)w[e].y * (double)acc[2 * e + 1];
    }
    __syncthreads();
    double* red = reinterpret_cast<double*>(sbase);
    red[tid] = valid ? d : 0.0;
    __syncthreads();
    if (valid && t == 0 && active) {
      double sum = 0.0;
      for (int e = 0; e < G::TS; ++e) sum += red[slot * G::TS + e];
      if (MODE == MODE_ENERGY) sum *= args.occ[k * args.n_occ + band];
      args.partial[split * args.split_stride + (size_t)k * args.n_own + band] = sum;
    }
  }

  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(tbase, S::TMEM_COLS);
}

}  // namespace hse
