// pairconv_tc.cuh - the Y and X stages of the fused pencil-load kernel on the tensor cores
// (tc_dft.cuh), for the split-precision option (kTcVariant, 24^3).  Included by
// pairconv_c64.cuh after the stage helpers it uses (Geo, Pencil).
//
// A warp's 32 pencils of a pass (whole warps: the ragged rule of the scalar stages) are two
// m16 tiles, carried through each stage together so that their load, scale, GEMM and store
// chains overlap.  Every lane's loads of both tiles complete before the first mma.sync that
// consumes them, which all lanes reach, so the results can then be stored in place.
#pragma once

#include "tc_dft.cuh"

namespace hse {

// Offsets of rows g and g + 8 of both tiles of the 32 pencils from p0 (YS: Y-stage pencils,
// else X-stage pencils).
template <int n, bool YS>
__device__ __forceinline__ void tc_tile_bases(int p0, int gq, int (&b0)[2], int (&b1)[2]) {
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const Pencil<n> pa(p0 + u * 16 + gq), pb(p0 + u * 16 + gq + 8);
    b0[u] = YS ? pa.ys : pa.xs;
    b1[u] = YS ? pb.ys : pb.xs;
  }
}

// Stage Y (DIR) of the thread's warp: the DFT of each Y pencil as a GEMM.
template <int n, int DIR, int PPT, int TS>
__device__ __forceinline__ void stage_y_tc(float2* g, int t, const TcTables<n>* tab) {
  using G = Geo<n>;
  using TG = TcGeo<n>;
  const int lane = threadIdx.x & 31, gq = lane >> 2;
  const uint4* W = DIR < 0 ? tab->fwd : tab->inv;
#pragma unroll 1
  for (int ps = 0; ps < PPT; ++ps) {
    if (TS * PPT != G::NN && t + ps * TS >= G::NN) break;  // whole warps past the last pencil
    int b0[2], b1[2];
    tc_tile_bases<n, true>((t - lane) + ps * TS, gq, b0, b1);
    uint32_t ah[2][TG::KS][4], al[2][TG::KS][4];
    float s0[2], s1[2], acc[2][TG::NT][4];
#pragma unroll
    for (int u = 0; u < 2; ++u) tc_load_a<n>(g, b0[u], b1[u], G::P, ah[u], al[u], s0[u], s1[u]);
    tc_gemm2<n>(acc, ah, al, W);
#pragma unroll
    for (int u = 0; u < 2; ++u) tc_store<n>(acc[u], s0[u], s1[u], g, b0[u], b1[u], G::P);
  }
}

// Stage X: forward DFT, multiply by the kernel row v * vscale (vrow: the pair's row of the
// kernel table, element (x, y, z) at x n^2 + y n + z), inverse DFT; the accumulators of the
// forward GEMM become the A fragments of the inverse one in registers.
template <int n, int PPT, int TS>
__device__ __forceinline__ void stage_x_tc(float2* g, int t, const TcTables<n>* tab, const float* __restrict__ vrow,
                                           float vscale) {
  using G = Geo<n>;
  using TG = TcGeo<n>;
  const int lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
#pragma unroll 1
  for (int ps = 0; ps < PPT; ++ps) {
    if (TS * PPT != G::NN && t + ps * TS >= G::NN) break;
    const int p0 = (t - lane) + ps * TS;
    int b0[2], b1[2];
    tc_tile_bases<n, false>(p0, gq, b0, b1);
    uint32_t ah[2][TG::KS][4], al[2][TG::KS][4];
    float s0[2], s1[2], acc[2][TG::NT][4];
#pragma unroll
    for (int u = 0; u < 2; ++u) tc_load_a<n>(g, b0[u], b1[u], G::Q, ah[u], al[u], s0[u], s1[u]);
    tc_gemm2<n>(acc, ah, al, tab->fwd);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      // the kernel values of this lane's accumulator elements (x index nt 4 + tq)
      const float* va = vrow + tq * G::NN + p0 + u * 16 + gq;
      const float r0 = vscale / (s0[u] * kTcWScale), r1 = vscale / (s1[u] * kTcWScale);
#pragma unroll
      for (int nt = 0; nt < TG::NT; ++nt) {
        const float wa = __ldg(va + nt * 4 * G::NN) * r0, wb = __ldg(va + nt * 4 * G::NN + 8) * r1;
        acc[u][nt][0] *= wa;
        acc[u][nt][1] *= wa;
        acc[u][nt][2] *= wb;
        acc[u][nt][3] *= wb;
      }
      tc_acc_to_a<n>(acc[u], ah[u], al[u], s0[u], s1[u]);
    }
    tc_gemm2<n>(acc, ah, al, tab->inv);
#pragma unroll
    for (int u = 0; u < 2; ++u) tc_store<n>(acc[u], s0[u], s1[u], g, b0[u], b1[u], G::Q);
  }
}

// One pair chain's Y and X stages on the tensor cores (vrow, vscale: the pair's kernel row
// and its scale times the occupation); all threads of the CTA call it together.
template <int n, int PPT, int TS>
__device__ __forceinline__ void pair_middle_tc(float2* g, int t, const TcTables<n>* tab, const float* vrow,
                                               float vscale, bool warp_on) {
  __syncthreads();
  if (warp_on) stage_y_tc<n, -1, PPT, TS>(g, t, tab);
  __syncthreads();
  if (warp_on) stage_x_tc<n, PPT, TS>(g, t, tab, vrow, vscale);
  __syncthreads();
  if (warp_on) stage_y_tc<n, +1, PPT, TS>(g, t, tab);
  __syncthreads();
}

}  // namespace hse
