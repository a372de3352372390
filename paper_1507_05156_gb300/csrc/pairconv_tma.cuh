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

// Shared and tensor memory of the staged kernel for pencil layout Lay (below).  TMEM columns
// of one warp: [acc (PPT pencils) | kernel rows (PPT) | owner u_i (PPT)].
template <int n, class Lay>
struct GeoS : StageGeo<n> {
  using G = Geo<n>;
  using SG = StageGeo<n>;
  static constexpr size_t GRIDS_BYTES = ((size_t)G::T * Lay::GRID_CPX * sizeof(float2) + 127) / 128 * 128;
  static constexpr int TAB = Lay::PPT * G::ROW;
  static constexpr int OWN = TAB + Lay::PPT * n;
  static constexpr int COLS_PER_WARP = OWN + Lay::PPT * G::ROW;
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
// stage (PPT), hence the block size, which pencils they are and how the smem grid is laid out;
// the pipeline is the same.
//   LayoutSeq:  two pencils per thread (t and t + n^2/2), transformed one after the other,
//               lanes on consecutive pencils, 64-bit smem accesses in Y and X.
//   LayoutOne:  one pencil per thread, twice the warps: with n^2 pencils per stage spread over
//               the four warp schedulers of an SM, the busiest scheduler carries fewer
//               pencil-passes than with LayoutSeq when n^2 / 128 has a small fractional part
//               (18^3: 3 instead of 4), and each scheduler has more warps to hide latency.
//   LayoutWide: two pencils per thread, neighbours in z in stages Y and X, so every smem access
//               moves both (128 bit) and both are transformed together (ILP).
// ---------------------------------------------------------------------------------------

template <int n, int PPT_>
struct LayoutLin {
  using G = Geo<n>;
  static constexpr int PPT = PPT_;
  static constexpr int TS = G::NN / PPT;                          // threads per owner slot
  static constexpr int THREADS = (G::T * TS + 31) / 32 * 32;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int GRID_CPX = G::GRID_CPX;
  static constexpr bool OK = G::ZFAST_Y == 1 && THREADS <= 1024;
  static __device__ __forceinline__ int zg(int t, int ps) { return Pencil<n>(t + ps * TS).zg; }
  static __device__ __forceinline__ void z_forward(float2* g, int t, bool valid, const float2* stg, uint32_t town) {
    stage_z_forward_staged<n, PPT>(g, t, valid, stg, town);
  }
  static __device__ __forceinline__ void z_inverse(const float2* g, int t, const float2* stg, uint32_t trow0) {
    stage_z_inverse_staged<n, PPT>(g, t, stg, trow0);
  }
  template <int DIR>
  static __device__ __forceinline__ void y(float2* g, int t, bool valid) {
    stage_y<n, DIR, PPT>(g, t, valid);
  }
  static __device__ __forceinline__ void x(float2* g, int t, bool valid, uint32_t ttab, float f) {
    stage_x<n, PPT>(g, t, valid, ttab, f);
  }
  static __device__ __forceinline__ void cache_row(int t, uint32_t ttab, const float* vrow, float scale) {
    cache_kernel_row<n, PPT>(t, ttab, vrow, scale);
  }
};

template <int n>
struct LayoutSeq : LayoutLin<n, 2> {};
template <int n>
struct LayoutOne : LayoutLin<n, 1> {};

// (P, Q, Z pairing) of the wide layout: 0 = (a, 2j), (a, 2j+1); 1 = (a, j), (a, j + n/2)
__host__ __device__ constexpr int wide_cfg(int n, int which) {
  return n == 4    ? (which == 0 ? 4 : which == 1 ? 20 : 0)
         : n == 6  ? (which == 0 ? 6 : which == 1 ? 38 : 0)
         : n == 8  ? (which == 0 ? 10 : which == 1 ? 88 : 1)
         : n == 10 ? (which == 0 ? 10 : which == 1 ? 106 : 0)
         : n == 12 ? (which == 0 ? 18 : which == 1 ? 220 : 1)
         : n == 18 ? (which == 0 ? 18 : which == 1 ? 338 : 1)
         : n == 20 ? (which == 0 ? 26 : which == 1 ? 532 : 1)
                   : -1;
}

template <int n>
struct LayoutWide {
  using G = Geo<n>;
  using S = StageGeo<n>;
  static constexpr int P = wide_cfg(n, 0), Q = wide_cfg(n, 1), ZM = wide_cfg(n, 2);
  static constexpr int H = n / 2;
  static constexpr int PPT = 2, TS = G::TS, THREADS = G::THREADS, WARPS = G::WARPS;
  static constexpr int GRID_CPX = n * (Q > 0 ? Q : 2);
  static constexpr bool OK = P > 0;
  // Z-stage pencil ps of thread t: (zx, zy)
  static __device__ __forceinline__ void zxy(int t, int ps, int& zx, int& zy) {
    const int a = t / H, j = t - a * H;
    zx = a;
    zy = ZM == 0 ? 2 * j + ps : j + ps * H;
  }
  static __device__ __forceinline__ int zg(int t, int ps) {
    int zx, zy;
    zxy(t, ps, zx, zy);
    return (zx * n + zy) * n;
  }
  static __device__ __forceinline__ void z_forward(float2* g, int t, bool valid, const float2* stg, uint32_t town) {
#pragma unroll 1
    for (int ps = 0; ps < 2; ++ps) {
      int zx, zy;
      zxy(t, ps, zx, zy);
      float uo[G::ROW];
      TmemRow<G::ROW>::load(town + (uint32_t)(ps * G::ROW), uo);
      const float4* s4 = reinterpret_cast<const float4*>(stg + (zx * n + zy) * S::SP);
      cpx<float> v[n];
#pragma unroll
      for (int e = 0; e < n / 2; ++e) {
        const float4 w = s4[e];
        v[2 * e] = {w.x * uo[4 * e] + w.y * uo[4 * e + 1], w.x * uo[4 * e + 1] - w.y * uo[4 * e]};
        v[2 * e + 1] = {w.z * uo[4 * e + 2] + w.w * uo[4 * e + 3], w.z * uo[4 * e + 3] - w.w * uo[4 * e + 2]};
      }
      fft<n, -1, float>(v);
      if (valid) store_s<n, 2>(v, g, zx * Q + zy * P, 1);
    }
  }
  static __device__ __forceinline__ void z_inverse(const float2* g, int t, const float2* stg, uint32_t trow0) {
#pragma unroll 1
    for (int ps = 0; ps < 2; ++ps) {
      int zx, zy;
      zxy(t, ps, zx, zy);
      cpx<float> v[n];
      load_s<n, 2>(v, g, zx * Q + zy * P, 1);
      fft<n, +1, float>(v);
      float acc[G::ROW];
      const uint32_t trow = trow0 + (uint32_t)(ps * G::ROW);
      TmemRow<G::ROW>::load(trow, acc);
      const float4* s4 = reinterpret_cast<const float4*>(stg + (zx * n + zy) * S::SP);
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
  // Y: pencils (x = t / H, z = 2 (t % H) + {0, 1}); one 128-bit access per element holds both
  template <int DIR>
  static __device__ __forceinline__ void y(float2* g, int t, bool valid) {
    const int ya = t / H, yp = t - ya * H;
    const int base = ya * Q + 2 * yp;
    cpx<float> a[n], b[n];
#pragma unroll
    for (int e = 0; e < n; ++e) {
      const float4 w = *reinterpret_cast<const float4*>(g + base + e * P);
      a[e] = {w.x, w.y};
      b[e] = {w.z, w.w};
    }
    fft<n, DIR, float>(a);
    fft<n, DIR, float>(b);
    if (valid) {
#pragma unroll
      for (int e = 0; e < n; ++e) *reinterpret_cast<float4*>(g + base + e * P) = make_float4(a[e].x, a[e].y, b[e].x, b[e].y);
    }
  }
  // X: pencils (y = t / H, z = 2 (t % H) + {0, 1}); kernel rows from the TMEM cache
  static __device__ __forceinline__ void x(float2* g, int t, bool valid, uint32_t ttab, float f) {
    const int ya = t / H, yp = t - ya * H;
    const int base = ya * P + 2 * yp;
    float ta[n], tb[n];
    TmemRow<n>::load(ttab, ta);
    TmemRow<n>::load(ttab + (uint32_t)n, tb);
    cpx<float> a[n], b[n];
#pragma unroll
    for (int e = 0; e < n; ++e) {
      const float4 w = *reinterpret_cast<const float4*>(g + base + e * Q);
      a[e] = {w.x, w.y};
      b[e] = {w.z, w.w};
    }
    fft<n, -1, float>(a);
    fft<n, -1, float>(b);
#pragma unroll
    for (int e = 0; e < n; ++e) {
      const float wa = ta[e] * f, wb = tb[e] * f;
      a[e].x *= wa;
      a[e].y *= wa;
      b[e].x *= wb;
      b[e].y *= wb;
    }
    fft<n, +1, float>(a);
    fft<n, +1, float>(b);
    if (valid) {
#pragma unroll
      for (int e = 0; e < n; ++e) *reinterpret_cast<float4*>(g + base + e * Q) = make_float4(a[e].x, a[e].y, b[e].x, b[e].y);
    }
  }
  static __device__ __forceinline__ void cache_row(int t, uint32_t ttab, const float* __restrict__ vrow, float scale) {
    const int ya = t / H, yp = t - ya * H;
    float ta[n], tb[n];
#pragma unroll
    for (int e = 0; e < n; ++e) {
      const float2 v = __ldg(reinterpret_cast<const float2*>(vrow + e * G::NN + ya * n + 2 * yp));
      ta[e] = v.x * scale;
      tb[e] = v.y * scale;
    }
    TmemRow<n>::store(ttab, ta);
    TmemRow<n>::store(ttab + (uint32_t)n, tb);
  }
};

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

// tmap: the partner array as rows of z-pencils, box {2 SP floats, BR rows}.  L: the pencil
// layout (LayoutSeq or LayoutWide).
template <int n, int MODE, template <int> class L>
__global__ void __launch_bounds__(L<n>::THREADS, 1)
    pairconv_tma_kernel(const PairArgs args, const __grid_constant__ CUtensorMap tmap) {
  using G = Geo<n>;
  using Lay = L<n>;
  using S = GeoS<n, Lay>;
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
  const bool valid = tid < G::T * Lay::TS;
  const int slot = valid ? tid / Lay::TS : 0;
  const int t = valid ? tid - slot * Lay::TS : 0;
  float2* grids = reinterpret_cast<float2*>(sbase);
  float2* g = grids + slot * Lay::GRID_CPX;
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
  for (int ps = 0; ps < Lay::PPT; ++ps) {
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

  uint32_t phase0 = 0, phase1 = 0;
  int buf = 0;
  int cur_kp = -1;
  while (q < npairs) {
    const int kp = kp_begin + q / args.n_part;
    const float f = item_occ(occ_sh, args, kp_begin, q);
    if (kp != cur_kp) {
      const int qrow = args.qidx[k * args.nk + kp];
      Lay::cache_row(t, ttab, args.vtab + (size_t)qrow * G::N, args.scale);
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
    Lay::z_forward(g, t, valid, stg, town);
    __syncthreads();
    // every thread is past its last read of stage[buf ^ 1]: refill it with the next partner
    const int qn = next_partner(occ_sh, args, kp_begin, q + 1, npairs);
    if (warp == 0 && qn < npairs && !abort_sh) {
      fence_proxy_async_smem();
      fill(qn, buf ^ 1);
    }
    Lay::template y<-1>(g, t, valid);
    __syncthreads();
    Lay::x(g, t, valid, ttab, f);
    __syncthreads();
    Lay::template y<+1>(g, t, valid);
    __syncthreads();
    Lay::z_inverse(g, t, stg, trow0);
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
    for (int ps = 0; ps < Lay::PPT; ++ps) {
      float acc[G::ROW];
      TmemRow<G::ROW>::load(trow0 + (uint32_t)(ps * G::ROW), acc);
      if (active) {
        float4* o = reinterpret_cast<float4*>(obase + Lay::zg(t, ps));
#pragma unroll
        for (int e = 0; e < n / 2; ++e) o[e] = make_float4(acc[4 * e], acc[4 * e + 1], acc[4 * e + 2], acc[4 * e + 3]);
      }
    }
  } else {
    const float2* lhs = (MODE == MODE_ENERGY) ? own : args.part2 + ((size_t)k * args.n_own + bandc) * G::N;
    double d = 0.0;
#pragma unroll 1
    for (int ps = 0; ps < Lay::PPT; ++ps) {
      float acc[G::ROW];
      TmemRow<G::ROW>::load(trow0 + (uint32_t)(ps * G::ROW), acc);
      cpx<float> w[n];
      load_pencil_global<n>(w, lhs + Lay::zg(t, ps));
#pragma unroll
      for (int e = 0; e < n; ++e) d += (double)w[e].x * (double)acc[2 * e] + (double)w[e].y * (double)acc[2 * e + 1];
    }
    __syncthreads();
    double* red = reinterpret_cast<double*>(sbase);
    red[tid] = valid ? d : 0.0;
    __syncthreads();
    if (valid && t == 0 && active) {
      double sum = 0.0;
      for (int e = 0; e < Lay::TS; ++e) sum += red[slot * Lay::TS + e];
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
