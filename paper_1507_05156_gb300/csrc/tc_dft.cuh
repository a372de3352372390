// tc_dft.cuh - length-n DFTs of a warp's 32 pencils on the tensor cores (mma.sync m16n8k16,
// FP16 operands, FP32 accumulation), for the split-precision option of the fused kernel: the Y
// and X axis transforms of the 3-D FFT of Sec. II C ("Fock": rho -> F -> x v -> F^-1) written
// as GEMMs.
//
// A pencil of n complex values is a row of 2n reals (re, im interleaved, as stored); the DFT
// y_k = sum_j x_j w^{jk} (w = exp(DIR 2 pi i / n)) is that row times the 2n x 2n real matrix
//   W[2j][2k] = cos t, W[2j+1][2k] = -sin t, W[2j][2k+1] = sin t, W[2j+1][2k+1] = cos t,
//   t = DIR 2 pi jk / n.
// A tile of 16 pencils is one m16 block; K = 2n in k-steps of 16, N = 2n in n-tiles of 8.
// FP32 data reaches FP16 precision in two halves: each row is scaled by a power of two that
// brings its largest magnitude to [2^14, 2^15), split into hi = fp16(x) and lo = fp16(x - hi),
// and W (scaled by 2^14) likewise; the three products hi*hi + hi*lo + lo*hi carry about 22
// significant bits (lo*lo, about 2^-22 of the result, is dropped), and the scales are divided
// out of the FP32 accumulators.
//
// Fragment layouts (m16n8k16, lane = 4 g + t): A holds rows g and g + 8, columns 2t, 2t + 1
// and 2t + 8, 2t + 9 -- with interleaved complex data, complex elements kk 8 + t and
// kk 8 + t + 4 of the two pencils; B holds rows (k) 2t, 2t + 1, 2t + 8, 2t + 9 of column
// (n) g; the accumulator holds rows g, g + 8, columns 2t, 2t + 1 of each n-tile -- complex
// element nt 4 + t.  The accumulators of n-tiles 2m, 2m + 1 are, element for element, the A
// fragment of k-step m, so a transform's output feeds the next transform without leaving
// registers.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "fft_reg.cuh"

namespace hse {

template <int n>
struct TcGeo {
  static_assert(n % 8 == 0, "2n must be a multiple of 16");
  static constexpr int KS = 2 * n / 16;  // k-steps
  static constexpr int NT = 2 * n / 8;   // n-tiles
  static constexpr int ENTRIES = KS * NT * 32;
};

// B fragments of W (forward and inverse) in shared memory, in fragment order: entry
// (kk, nt, lane) = {hi(b0, b1), hi(b2, b3), lo(b0, b1), lo(b2, b3)}.
template <int n>
struct TcTables {
  uint4 fwd[TcGeo<n>::ENTRIES];
  uint4 inv[TcGeo<n>::ENTRIES];
};

__device__ __forceinline__ uint32_t pack_half2(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// hi and lo halves of a, b (already scaled into the FP16 range)
__device__ __forceinline__ void split_half2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 hf = __half22float2(h);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = pack_half2(a - hf.x, b - hf.y);
}

constexpr float kTcWScale = 16384.f;  // 2^14

// cos and sin of 2 pi m / n, m < n, rounded to FP32 at compile time
template <int n>
struct TcTrig {
  float c[n], s[n];
};
template <int n>
constexpr TcTrig<n> make_tc_trig() {
  TcTrig<n> t{};
  for (int m = 0; m < n; ++m) {
    t.c[m] = (float)trig2pi(m, n, 0);
    t.s[m] = (float)trig2pi(m, n, 1);
  }
  return t;
}
template <int n>
__device__ const TcTrig<n> kTcTrig = make_tc_trig<n>();

// W[K][N] (real form above), times 2^14
template <int n, int DIR>
__device__ __forceinline__ float tc_w(int K, int N) {
  const int j = K >> 1, c = K & 1, k = N >> 1, d = N & 1;
  const int jk = (j * k) % n;
  const float cs = kTcTrig<n>.c[jk], sn = DIR * kTcTrig<n>.s[jk];
  const float w = (c == d) ? cs : (c == 0 ? sn : -sn);
  return w * kTcWScale;
}

// Fill both tables (all threads of the block; a barrier must follow).
template <int n>
__device__ void tc_build_tables(TcTables<n>* tab) {
  using TG = TcGeo<n>;
  for (int e = threadIdx.x; e < TG::ENTRIES; e += blockDim.x) {
    const int lane = e & 31, nt = (e >> 5) % TG::NT, kk = (e >> 5) / TG::NT;
    const int g = lane >> 2, t = lane & 3;
    const int K0 = kk * 16 + 2 * t, N0 = nt * 8 + g;
    uint4 f, v;
    split_half2(tc_w<n, -1>(K0, N0), tc_w<n, -1>(K0 + 1, N0), f.x, f.z);
    split_half2(tc_w<n, -1>(K0 + 8, N0), tc_w<n, -1>(K0 + 9, N0), f.y, f.w);
    split_half2(tc_w<n, +1>(K0, N0), tc_w<n, +1>(K0 + 1, N0), v.x, v.z);
    split_half2(tc_w<n, +1>(K0 + 8, N0), tc_w<n, +1>(K0 + 9, N0), v.y, v.w);
    tab->fwd[e] = f;
    tab->inv[e] = v;
  }
}

__device__ __forceinline__ void mma_f16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Power-of-two scale bringing m (> 0) to [2^14, 2^15); 1 for m == 0.  Capped at 2^110 (rows
// below 2^-95 in magnitude), so that the scale times 2^14 stays finite in FP32.
__device__ __forceinline__ float tc_row_scale(float m) {
  if (!(m > 0.f)) return 1.f;
  int e = 0;
  frexpf(m, &e);
  return ldexpf(1.f, 15 - max(e, -95));
}

// max over the 4 lanes of a fragment row group (lanes 4g .. 4g + 3)
__device__ __forceinline__ float quad_max(float v) {
  v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 1));
  v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 2));
  return v;
}

// acc = (scaled A: hi, lo per k-step) x W, for every n-tile
template <int n>
__device__ __forceinline__ void tc_gemm(float (&acc)[TcGeo<n>::NT][4], const uint32_t (&ah)[TcGeo<n>::KS][4],
                                        const uint32_t (&al)[TcGeo<n>::KS][4], const uint4* __restrict__ tab) {
  using TG = TcGeo<n>;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int nt = 0; nt < TG::NT; ++nt) {
    acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < TG::KS; ++kk) {
      const uint4 b = tab[(kk * TG::NT + nt) * 32 + lane];
      mma_f16(acc[nt], ah[kk], b.x, b.y);
      mma_f16(acc[nt], ah[kk], b.z, b.w);
      mma_f16(acc[nt], al[kk], b.x, b.y);
    }
  }
}

// The same for two tiles at once (independent accumulator chains interleaved, each B
// fragment loaded once for both).
template <int n>
__device__ __forceinline__ void tc_gemm2(float (&acc)[2][TcGeo<n>::NT][4], const uint32_t (&ah)[2][TcGeo<n>::KS][4],
                                         const uint32_t (&al)[2][TcGeo<n>::KS][4], const uint4* __restrict__ tab) {
  using TG = TcGeo<n>;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int nt = 0; nt < TG::NT; ++nt) {
#pragma unroll
    for (int u = 0; u < 2; ++u) acc[u][nt][0] = acc[u][nt][1] = acc[u][nt][2] = acc[u][nt][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < TG::KS; ++kk) {
      const uint4 b = tab[(kk * TG::NT + nt) * 32 + lane];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        mma_f16(acc[u][nt], ah[u][kk], b.x, b.y);
        mma_f16(acc[u][nt], ah[u][kk], b.z, b.w);
        mma_f16(acc[u][nt], al[u][kk], b.x, b.y);
      }
    }
  }
}

// Accumulators (rows g, g + 8 in [0..1] / [2..3] of each n-tile) -> scaled split A fragments.
// Returns the two rows' scales in s0 (row g) and s1 (row g + 8).
template <int n>
__device__ __forceinline__ void tc_acc_to_a(const float (&acc)[TcGeo<n>::NT][4], uint32_t (&ah)[TcGeo<n>::KS][4],
                                            uint32_t (&al)[TcGeo<n>::KS][4], float& s0, float& s1) {
  using TG = TcGeo<n>;
  float m0 = 0.f, m1 = 0.f;
#pragma unroll
  for (int nt = 0; nt < TG::NT; ++nt) {
    m0 = fmaxf(m0, fmaxf(fabsf(acc[nt][0]), fabsf(acc[nt][1])));
    m1 = fmaxf(m1, fmaxf(fabsf(acc[nt][2]), fabsf(acc[nt][3])));
  }
  s0 = tc_row_scale(quad_max(m0));
  s1 = tc_row_scale(quad_max(m1));
#pragma unroll
  for (int m = 0; m < TG::KS; ++m) {
    split_half2(acc[2 * m][0] * s0, acc[2 * m][1] * s0, ah[m][0], al[m][0]);
    split_half2(acc[2 * m][2] * s1, acc[2 * m][3] * s1, ah[m][1], al[m][1]);
    split_half2(acc[2 * m + 1][0] * s0, acc[2 * m + 1][1] * s0, ah[m][2], al[m][2]);
    split_half2(acc[2 * m + 1][2] * s1, acc[2 * m + 1][3] * s1, ah[m][3], al[m][3]);
  }
}

// Rows of a 16-pencil tile from shared memory (pencil r of the tile starts at base[r], element
// stride `stride` float2) -> scaled split A fragments; s0 / s1: the scales of rows g / g + 8.
template <int n>
__device__ __forceinline__ void tc_load_a(const float2* g_s, int base0, int base1, int stride,
                                          uint32_t (&ah)[TcGeo<n>::KS][4], uint32_t (&al)[TcGeo<n>::KS][4],
                                          float& s0, float& s1) {
  using TG = TcGeo<n>;
  const int t = threadIdx.x & 3;
  float2 x[TG::KS][4];
  float m0 = 0.f, m1 = 0.f;
#pragma unroll
  for (int kk = 0; kk < TG::KS; ++kk) {
    const int j = kk * 8 + t;
    x[kk][0] = g_s[base0 + j * stride];
    x[kk][1] = g_s[base1 + j * stride];
    x[kk][2] = g_s[base0 + (j + 4) * stride];
    x[kk][3] = g_s[base1 + (j + 4) * stride];
    m0 = fmaxf(m0, fmaxf(fmaxf(fabsf(x[kk][0].x), fabsf(x[kk][0].y)), fmaxf(fabsf(x[kk][2].x), fabsf(x[kk][2].y))));
    m1 = fmaxf(m1, fmaxf(fmaxf(fabsf(x[kk][1].x), fabsf(x[kk][1].y)), fmaxf(fabsf(x[kk][3].x), fabsf(x[kk][3].y))));
  }
  s0 = tc_row_scale(quad_max(m0));
  s1 = tc_row_scale(quad_max(m1));
#pragma unroll
  for (int kk = 0; kk < TG::KS; ++kk) {
    split_half2(x[kk][0].x * s0, x[kk][0].y * s0, ah[kk][0], al[kk][0]);
    split_half2(x[kk][1].x * s1, x[kk][1].y * s1, ah[kk][1], al[kk][1]);
    split_half2(x[kk][2].x * s0, x[kk][2].y * s0, ah[kk][2], al[kk][2]);
    split_half2(x[kk][3].x * s1, x[kk][3].y * s1, ah[kk][3], al[kk][3]);
  }
}

// Accumulators / (scale 2^14) -> the rows in shared memory (complex element nt 4 + t).
template <int n>
__device__ __forceinline__ void tc_store(const float (&acc)[TcGeo<n>::NT][4], float s0, float s1, float2* g_s,
                                         int base0, int base1, int stride) {
  using TG = TcGeo<n>;
  const int t = threadIdx.x & 3;
  const float r0 = 1.f / (s0 * kTcWScale), r1 = 1.f / (s1 * kTcWScale);
#pragma unroll
  for (int nt = 0; nt < TG::NT; ++nt) {
    const int k = nt * 4 + t;
    g_s[base0 + k * stride] = make_float2(acc[nt][0] * r0, acc[nt][1] * r0);
    g_s[base1 + k * stride] = make_float2(acc[nt][2] * r1, acc[nt][3] * r1);
  }
}

}  // namespace hse
