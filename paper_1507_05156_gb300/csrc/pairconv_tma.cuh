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
//   LayoutSplit: one pencil per thread for the first R = 128 floor(n^2 / 128) pencils (whole
//                warps, the same count on every scheduler), plus four warps, one per scheduler,
//                that transform the L = n^2 - R pencils left over with their DFT split over
//                lanes (below), L / 4 each.  For 20^3 (R = 384, L = 16) this replaces a thirteenth
//                warp, which gave one scheduler four full pencil passes per stage against three
//                on the others, by warps whose pass costs a fraction of one and runs beside the
//                regular ones.
// TMEM columns of a warp: [acc (PPT pencils) | kernel rows (PPT) | owner u_i (PPT) | extra].
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
  static constexpr int COLS_PER_WARP = OWN + PPT * G::ROW;
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
  // pencils beyond the regular ones (LayoutSplit): none here
  static __device__ __forceinline__ bool regular(int) { return true; }
  static __device__ __forceinline__ void extra_init(int, const float2*, uint32_t) {}
  static __device__ __forceinline__ void extra_store(int, float2*, uint32_t, bool) {}
  static __device__ __forceinline__ double extra_dot(int, const float2*, uint32_t) { return 0.0; }
};

template <int n>
struct LayoutSeq : LayoutLin<n, 2> {};
template <int n>
struct LayoutOne : LayoutLin<n, 1> {};

// --- DFT of one pencil split over lanes (prime-factor form, Sec. "Good-Thomas") -------------
// n = N1 N2 with gcd(N1, N2) = 1.  With posA(a, b) = (N2 a + N1 b) mod n and
// crt(k1, k2) the k with k = k1 (mod N1), k = k2 (mod N2), the DFT X[crt(k1, k2)] =
// sum_b w_N2^(b k2) sum_a w_N1^(a k1) x[posA(a, b)] splits into
//   pass A: for each b (one lane), the N1-point DFT over a, written back to posA(k1, b);
//   pass B: for each k1 (one lane), the N2-point DFT over b of the values at posA(k1, b),
//           written to crt(k1, k2).
// When N2 = 1 (mod N1) the positions a lane reads in pass B are the ones it writes, so every
// pass works in place on a set of positions no other lane of the pass touches.
__host__ __device__ constexpr int inv_mod_c(int a, int m) {
  int x = 1;
  while ((a * x) % m != 1 % m) ++x;
  return x;
}

template <int n>
struct SplitGeo {
  static constexpr int N1 = pfa_n1(n);
  static constexpr int N2 = N1 > 0 ? n / N1 : 1;
  static constexpr int NN = n * n;
  static constexpr int R = NN / 128 * 128;                 // regular pencils (whole warps)
  static constexpr int L = NN - R;                         // split pencils
  static constexpr int PER = L / 4;                        // split pencils per scheduler
  static constexpr int E1 = N1 > 1 ? (N2 * inv_mod_c(N2 % N1, N1)) % n : 0;
  static constexpr int E2 = N1 > 1 ? (N1 * inv_mod_c(N1 % N2, N2)) % n : 0;
  static constexpr bool OK = N1 > 1 && R > 0 && L > 0 && L % 4 == 0 && PER * N2 <= 32 && N2 % N1 == 1 &&
                             Geo<n>::T == 1 && Geo<n>::ZFAST_Y == 1;
  static constexpr int HOST0 = R / 32;                     // warps HOST0 .. HOST0 + 3 take them
  // extra TMEM columns of a hosting lane: owner u_i at its pass-A positions (2 N1 floats),
  // accumulator there (2 N1), kernel values at its pass-B positions (N2, padded)
  static constexpr int C_OWN = 0, C_ACC = 2 * N1, C_KER = 4 * N1;
  static constexpr int KW = N2 <= 4 ? 4 : (N2 <= 6 ? 6 : 8);
  static constexpr int COLS = (4 * N1 + KW + 7) / 8 * 8;
  static __host__ __device__ __forceinline__ int posA(int a, int b) {  // a, b < n: one wrap at most
    const int v = N2 * a + N1 * b;
    return v >= n ? v - n : v;
  }
  static __host__ __device__ __forceinline__ int crt(int k1e1, int k2) {  // k1e1 = (k1 E1) mod n
    const int v = k1e1 + (k2 * E2) % n;
    return v >= n ? v - n : v;
  }
};

template <int n>
struct LayoutSplit {
  using G = Geo<n>;
  using SG = SplitGeo<n>;
  using S = StageGeo<n>;
  static constexpr int PPT = 1;
  static constexpr int TS = SG::OK ? SG::R + 128 : G::NN;
  static constexpr int THREADS = TS, WARPS = TS / 32;
  static constexpr int GRID_CPX = G::GRID_CPX;
  static constexpr bool OK = SG::OK && THREADS <= 1024;
  static constexpr int TAB = G::ROW;
  static constexpr int OWN = TAB + n;
  static constexpr int EXTRA = OWN + G::ROW;
  static constexpr int COLS_PER_WARP = EXTRA + SG::COLS;
  // the regular pencils 0 .. R-1 (pencil = thread in every stage: with the split pencils
  // beside them, the bank-spread X order measured slower, 35.3 against 34.7 ms at 20^3)
  using Reg = LayoutLin<n, 1, false>;
  static __device__ __forceinline__ bool regular(int t) { return t < SG::R; }
  // block barriers only
  static constexpr bool GROUPED = false;
  static __device__ __forceinline__ void group_sync(int) {}

  // role of this lane in the hosting warp: s = scheduler, A: (pencil, b), B: (pencil, k1)
  struct Roles {
    bool host, a_on, b_on;
    int pa, b, pb, k1, k1e1;
    __device__ __forceinline__ explicit Roles(int t) {
      const int warp = t >> 5, lane = t & 31;
      host = warp >= SG::HOST0;
      const int first = SG::R + (warp - SG::HOST0) * SG::PER;
      a_on = host && lane < SG::PER * SG::N2;
      b_on = host && lane < SG::PER * SG::N1;
      // lanes without a role keep an in-range pencil (its index also selects table entries)
      pa = a_on ? first + lane / SG::N2 : SG::R;
      b = lane % SG::N2;
      pb = b_on ? first + lane / SG::N1 : SG::R;
      k1 = lane % SG::N1;
      k1e1 = (k1 * SG::E1) % n;
    }
  };

  template <int DIR>
  static __device__ __forceinline__ void pass_a(float2* g, int base, int stride, int b) {
    cpx<float> v[SG::N1];
#pragma unroll
    for (int a = 0; a < SG::N1; ++a) {
      const float2 w = g[base + SG::posA(a, b) * stride];
      v[a] = {w.x, w.y};
    }
    fft<SG::N1, DIR, float>(v);
#pragma unroll
    for (int a = 0; a < SG::N1; ++a) g[base + SG::posA(a, b) * stride] = make_float2(v[a].x, v[a].y);
  }
  template <int DIR>
  static __device__ __forceinline__ void pass_b(float2* g, int base, int stride, int k1, int k1e1) {
    cpx<float> v[SG::N2];
#pragma unroll
    for (int b = 0; b < SG::N2; ++b) {
      const float2 w = g[base + SG::posA(k1, b) * stride];
      v[b] = {w.x, w.y};
    }
    fft<SG::N2, DIR, float>(v);
#pragma unroll
    for (int k2 = 0; k2 < SG::N2; ++k2) g[base + SG::crt(k1e1, k2) * stride] = make_float2(v[k2].x, v[k2].y);
  }

  static __device__ __forceinline__ int zg(int t, int ps) { return Reg::zg(t, ps); }

  static __device__ __forceinline__ void z_forward(float2* g, int t, bool valid, const float2* stg, uint32_t trow0) {
    const Roles r(t);
    if (r.host) {  // warp-uniform
      float uo[2 * SG::N1];
      TmemRow<2 * SG::N1>::load(trow0 + (uint32_t)(EXTRA + SG::C_OWN), uo);
      if (r.a_on) {
        const Pencil<n> pc(r.pa);
        const float2* srow = stg + (pc.zg / n) * S::SP;
        cpx<float> v[SG::N1];
#pragma unroll
        for (int a = 0; a < SG::N1; ++a) {
          const float2 w = srow[SG::posA(a, r.b)];
          v[a] = {w.x * uo[2 * a] + w.y * uo[2 * a + 1], w.x * uo[2 * a + 1] - w.y * uo[2 * a]};
        }
        fft<SG::N1, -1, float>(v);
#pragma unroll
        for (int a = 0; a < SG::N1; ++a) g[pc.zs + SG::posA(a, r.b)] = make_float2(v[a].x, v[a].y);
      }
      __syncwarp();
      if (r.b_on) pass_b<-1>(g, Pencil<n>(r.pb).zs, 1, r.k1, r.k1e1);
    }
    if (regular(t)) Reg::z_forward(g, t, valid, stg, trow0);
  }

  template <int DIR>
  static __device__ __forceinline__ void y(float2* g, int t, bool valid) {
    const Roles r(t);
    if (r.host) {
      if (r.a_on) pass_a<DIR>(g, Pencil<n>(r.pa).ys, G::P, r.b);
      __syncwarp();
      if (r.b_on) pass_b<DIR>(g, Pencil<n>(r.pb).ys, G::P, r.k1, r.k1e1);
    }
    if (regular(t)) Reg::template y<DIR>(g, t, valid);
  }

  static __device__ __forceinline__ void x(float2* g, int t, bool valid, uint32_t trow0, float f) {
    const Roles r(t);
    if (r.host) {
      float kv[SG::KW];
      TmemRow<SG::KW>::load(trow0 + (uint32_t)(EXTRA + SG::C_KER), kv);
      const int xa = Pencil<n>(r.pa).xs;
      if (r.a_on) pass_a<-1>(g, xa, G::Q, r.b);
      __syncwarp();
      if (r.b_on) {
        const int base = Pencil<n>(r.pb).xs;
        cpx<float> v[SG::N2];
#pragma unroll
        for (int b = 0; b < SG::N2; ++b) {
          const float2 w = g[base + SG::posA(r.k1, b) * G::Q];
          v[b] = {w.x, w.y};
        }
        fft<SG::N2, -1, float>(v);  // v[k2] = X[crt(k1, k2)]
#pragma unroll
        for (int k2 = 0; k2 < SG::N2; ++k2) {
          const float w = kv[k2] * f;
          v[k2].x *= w;
          v[k2].y *= w;
        }
        fft<SG::N2, +1, float>(v);  // back to b, still at fixed k1
#pragma unroll
        for (int b = 0; b < SG::N2; ++b) g[base + SG::posA(r.k1, b) * G::Q] = make_float2(v[b].x, v[b].y);
      }
      __syncwarp();
      if (r.a_on) pass_a<+1>(g, xa, G::Q, r.b);
    }
    if (regular(t)) Reg::x(g, t, valid, trow0, f);
  }

  static __device__ __forceinline__ void z_inverse(const float2* g_, int t, const float2* stg, uint32_t trow0) {
    const Roles r(t);
    if (r.host) {
      float2* g = const_cast<float2*>(g_);  // the split pencils pass through the grid in place
      if (r.b_on) {
        // natural order -> (k1, b): inverse N2-point DFTs first, in place on the lane's set
        const int base = Pencil<n>(r.pb).zs;
        cpx<float> v[SG::N2];
#pragma unroll
        for (int k2 = 0; k2 < SG::N2; ++k2) {
          const float2 w = g[base + SG::crt(r.k1e1, k2)];
          v[k2] = {w.x, w.y};
        }
        fft<SG::N2, +1, float>(v);
#pragma unroll
        for (int b = 0; b < SG::N2; ++b) g[base + SG::posA(r.k1, b)] = make_float2(v[b].x, v[b].y);
      }
      __syncwarp();
      float acc[2 * SG::N1];
      const uint32_t tacc = trow0 + (uint32_t)(EXTRA + SG::C_ACC);
      TmemRow<2 * SG::N1>::load(tacc, acc);
      if (r.a_on) {
        const Pencil<n> pc(r.pa);
        cpx<float> v[SG::N1];
#pragma unroll
        for (int a = 0; a < SG::N1; ++a) {
          const float2 w = g[pc.zs + SG::posA(a, r.b)];
          v[a] = {w.x, w.y};
        }
        fft<SG::N1, +1, float>(v);  // v[a] = phi at posA(a, b)
        const float2* srow = stg + (pc.zg / n) * S::SP;
#pragma unroll
        for (int a = 0; a < SG::N1; ++a) {
          const float2 w = srow[SG::posA(a, r.b)];
          acc[2 * a] = fmaf(w.x, v[a].x, fmaf(-w.y, v[a].y, acc[2 * a]));
          acc[2 * a + 1] = fmaf(w.x, v[a].y, fmaf(w.y, v[a].x, acc[2 * a + 1]));
        }
      }
      TmemRow<2 * SG::N1>::store(tacc, acc);
      __syncwarp();  // the next pair's Z forward rewrites these positions from other lanes
    }
    if (regular(t)) Reg::z_inverse(g_, t, stg, trow0);
  }

  static __device__ __forceinline__ void cache_row(int t, uint32_t trow0, const float* __restrict__ vrow, float scale) {
    const Roles r(t);
    if (r.host) {
      float kv[SG::KW];
#pragma unroll
      for (int k2 = 0; k2 < SG::KW; ++k2)
        kv[k2] = (r.b_on && k2 < SG::N2) ? __ldg(vrow + SG::crt(r.k1e1, k2) * G::NN + r.pb) * scale
                                         : 0.f;
      TmemRow<SG::KW>::store(trow0 + (uint32_t)(EXTRA + SG::C_KER), kv);
    }
    if (regular(t)) Reg::cache_row(t, trow0, vrow, scale);
  }

  static __device__ __forceinline__ void extra_init(int t, const float2* own, uint32_t trow0) {
    const Roles r(t);
    if (!r.host) return;
    float w[2 * SG::N1], z[2 * SG::N1];
    const int zg0 = Pencil<n>(r.pa).zg;
#pragma unroll
    for (int a = 0; a < SG::N1; ++a) {
      const float2 u = r.a_on ? __ldg(own + zg0 + SG::posA(a, r.b)) : make_float2(0.f, 0.f);
      w[2 * a] = u.x;
      w[2 * a + 1] = u.y;
      z[2 * a] = z[2 * a + 1] = 0.f;
    }
    TmemRow<2 * SG::N1>::store(trow0 + (uint32_t)(EXTRA + SG::C_OWN), w);
    TmemRow<2 * SG::N1>::store(trow0 + (uint32_t)(EXTRA + SG::C_ACC), z);
  }
  static __device__ __forceinline__ void extra_store(int t, float2* obase, uint32_t trow0, bool active) {
    const Roles r(t);
    if (!r.host) return;
    float acc[2 * SG::N1];
    TmemRow<2 * SG::N1>::load(trow0 + (uint32_t)(EXTRA + SG::C_ACC), acc);
    if (active && r.a_on) {
      const int zg0 = Pencil<n>(r.pa).zg;
#pragma unroll
      for (int a = 0; a < SG::N1; ++a) obase[zg0 + SG::posA(a, r.b)] = make_float2(acc[2 * a], acc[2 * a + 1]);
    }
  }
  static __device__ __forceinline__ double extra_dot(int t, const float2* lhs, uint32_t trow0) {
    const Roles r(t);
    if (!r.host) return 0.0;
    float acc[2 * SG::N1];
    TmemRow<2 * SG::N1>::load(trow0 + (uint32_t)(EXTRA + SG::C_ACC), acc);
    double d = 0.0;
    if (r.a_on) {
      const int zg0 = Pencil<n>(r.pa).zg;
#pragma unroll
      for (int a = 0; a < SG::N1; ++a) {
        const float2 w = __ldg(lhs + zg0 + SG::posA(a, r.b));
        d += (double)w.x * (double)acc[2 * a] + (double)w.y * (double)acc[2 * a + 1];
      }
    }
    return d;
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

  const int per_split = args.nk_own * args.ntiles;
  const int split = item / per_split;
  const int rem = item - split * per_split;
  const int k = rem / args.ntiles;
  const int band = (rem - k * args.ntiles) * G::T + slot;
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
  const bool reg = on && Lay::regular(t);  // warp-uniform
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
  if (on) Lay::extra_init(t, own, trow0);

  int buf = 0;
  int cur_kp = -1;
  while (q < npairs) {
    const int kp = kp_begin + q / args.n_part;
    const float f = item_occ(sh.occ, args, kp_begin, q);
    if (kp != cur_kp) {
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

  if constexpr (MODE == MODE_APPLY) {
    float2* obase = args.out + split * args.split_stride + ((size_t)k * args.n_own + bandc) * G::N;
#pragma unroll 1
    for (int ps = 0; ps < (reg ? Lay::PPT : 0); ++ps) {
      float acc[G::ROW];
      TmemRow<G::ROW>::load(trow0 + (uint32_t)(ps * G::ROW), acc);
      if (active) {
        float4* o = reinterpret_cast<float4*>(obase + Lay::zg(t, ps));
#pragma unroll
        for (int e = 0; e < n / 2; ++e) o[e] = make_float4(acc[4 * e], acc[4 * e + 1], acc[4 * e + 2], acc[4 * e + 3]);
      }
    }
    if (on) Lay::extra_store(t, obase, trow0, active);
  } else {
    const float2* lhs = (MODE == MODE_ENERGY) ? own : args.part2 + ((size_t)k * args.n_own + bandc) * G::N;
    double d = 0.0;
#pragma unroll 1
    for (int ps = 0; ps < (reg ? Lay::PPT : 0); ++ps) {
      float acc[G::ROW];
      TmemRow<G::ROW>::load(trow0 + (uint32_t)(ps * G::ROW), acc);
      cpx<float> w[n];
      load_pencil_global<n>(w, lhs + Lay::zg(t, ps));
#pragma unroll
      for (int e = 0; e < n; ++e) d += (double)w[e].x * (double)acc[2 * e] + (double)w[e].y * (double)acc[2 * e + 1];
    }
    if (on) d += Lay::extra_dot(t, lhs, trow0);
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

// One work item per CTA.  L: the pencil layout (LayoutSeq, LayoutOne or LayoutSplit).
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
