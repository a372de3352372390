// pairconv_c64.cuh - fused FP32 (complex64) pair-convolution kernel of the Fock-like term.
//
// One CTA owns a tile of T "owner" orbitals at one k-point and loops over every partner
// (k', j).  For each pair it runs the whole chain of Sec. II C, Eq. "Fock" / "Fock-DS"
// with the pair's grid resident in shared memory:
//
//   Z: pair density rho = conj(u_j) u_i on z-pencils (registers), FFT along z
//   Y: FFT along y                     (smem -> registers -> smem)
//   X: FFT along x, multiply by v(|G+q|) * s / N, inverse FFT along x
//   Y: inverse FFT along y
//   Z: inverse FFT along z, multiply by the partner and accumulate (epilogue)
//
// Each thread owns two pencils per stage and transforms them one after the other (so only
// one pencil is live in registers and two CTAs fit per SM at 20^3); in every stage the
// lanes of a warp take consecutive pencils.  The shared grid is interleaved complex,
// G[x*Q + y*P + z], with pitches P, Q chosen by an offline search of the bank mapping of
// all four transposes.  The owner's accumulator lives in Tensor Memory (one TMEM lane per
// thread, 2 x 2n columns) for the whole partner loop and is written to HBM once.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda_bf16.h>

#include "fft_reg.cuh"
#include "tmem.cuh"
#include "tmem_gen.cuh"

namespace hse {

// Per grid side: pitches (complex units), Z-stage lane order (zfast_y: lanes run along y,
// else along x), Z-stage access width in complex values (1: 64 bit, 2: 128 bit), owner
// orbitals per CTA.
struct KCfg {
  int P, Q, zfast_y, zvec, slots;
};

__host__ __device__ constexpr KCfg kcfg(int n) {
  return n == 4    ? KCfg{4, 22, 1, 2, 32}
         : n == 6  ? KCfg{6, 38, 1, 2, 16}
         : n == 8  ? KCfg{9, 72, 1, 1, 8}
         : n == 10 ? KCfg{10, 106, 1, 2, 4}
         : n == 12 ? KCfg{12, 156, 1, 2, 4}
         : n == 16 ? KCfg{17, 272, 1, 1, 2}
         : n == 18 ? KCfg{18, 338, 1, 2, 1}
         : n == 20 ? KCfg{21, 420, 1, 1, 1}
         : n == 24 ? KCfg{25, 600, 1, 1, 1}
                   : KCfg{0, 0, 0, 0, 0};
}

__host__ __device__ constexpr int slots_for(int n) { return kcfg(n).slots; }
// complex elements of one orbital in the pencil-blocked layout (OrbBlk below)
__host__ __device__ constexpr size_t blocked_stride(int n) { return (size_t)((n * n + 31) / 32) * 32 * n; }

__host__ __device__ constexpr int pow2_at_least(int x) {
  int p = 32;
  while (p < x) p *= 2;
  return p;
}

template <int n>
struct Geo {
  static constexpr KCfg C = kcfg(n);
  static_assert(C.P > 0 && n % 2 == 0, "fused form needs an even grid side from the supported set");
  static constexpr int P = C.P, Q = C.Q, ZFAST_Y = C.zfast_y, ZVEC = C.zvec, T = C.slots;
  static constexpr int H = n / 2;
  static constexpr int NN = n * n;
  static constexpr int N = n * n * n;
  static constexpr int TS = n * H;                                // threads per owner slot (2 pencils each)
  static constexpr int THREADS = ((T * TS + 31) / 32) * 32;       // whole warps (TMEM ops are warp-wide)
  static constexpr int WARPS = THREADS / 32;
  static constexpr int GRID_CPX = n * Q;                          // complex slots of one slot's grid
  static constexpr int ROW = 2 * n;                               // floats of one pencil's accumulator
  static constexpr int TAB = 2 * ROW;                             // column of the kernel-row cache
  static constexpr int COLS_PER_WARP = 2 * ROW + 2 * n;           // 2 accumulators + 2 kernel rows
  static constexpr int TMEM_COLS = pow2_at_least(((WARPS + 3) / 4) * COLS_PER_WARP);
  static constexpr size_t SMEM_BYTES = (size_t)T * GRID_CPX * sizeof(float2);
  static_assert(TMEM_COLS <= 512, "accumulator exceeds tensor memory");
  // two CTAs per SM are possible when tensor memory and shared memory allow it; the
  // 2-CTA variant caps registers (per-SMSP register file), the 1-CTA variant does not
  static constexpr int MAXB = (512 / TMEM_COLS >= 2 && 2 * (SMEM_BYTES + 1024) <= 233472) ? 2 : 1;
  static_assert(ZVEC == 1 || (P % 2 == 0 && Q % 2 == 0), "128-bit Z accesses need even pitches");
};

// Thread and TMEM geometry of the pencil-load pipeline with TS threads per owner slot, each
// taking pencils t, t + TS, ... (at most PPT of them) in every stage; PPT = 2 with TS = n^2/2
// is Geo's own.  TS need not divide n^2 (24^3: 384 threads, the first 192 take a second
// pencil), but n^2 - (PPT - 1) TS must be a multiple of 32 so that the last pass covers whole
// warps.
template <int n, int PPT, int TS_ = Geo<n>::NN / PPT>
struct GeoP {
  using G = Geo<n>;
  static constexpr int TS = TS_;                                  // threads per owner slot
  static_assert((PPT - 1) * TS < G::NN && PPT * TS >= G::NN, "PPT passes of TS threads cover the pencils");
  static constexpr int THREADS = ((G::T * TS + 31) / 32) * 32;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int TAB = PPT * G::ROW;                        // column of the kernel-row cache
  static constexpr int COLS_PER_WARP = PPT * G::ROW + PPT * n;    // accumulators + kernel rows
  static constexpr int TMEM_COLS = pow2_at_least(((WARPS + 3) / 4) * COLS_PER_WARP);
};

// What a launch computes.
enum PairMode : int {
  MODE_APPLY = 0,   // owner = target i, partner = occupied j: out = V_x u_i
  MODE_ENERGY = 1,  // as APPLY, epilogue: partial[owner] = f_i Re<u_i, V_x u_i> (FP64)
  MODE_DOT = 2,     // as APPLY, epilogue: partial[owner] = Re<ybar_i, (V u)_i> (FP64)
  MODE_OCC = 3,     // owner = occupied j, partners = (u_i, ybar_i): VJP w.r.t. u_occ
};

struct PairArgs {
  const float2* own;    // [nk][n_own][N]  owner orbitals
  const float2* part;   // [nk][n_part][N] partner orbitals (u_occ for APPLY, u_tgt for OCC)
  const float2* part2;  // MODE_OCC: ybar [nk][n_part][N];  MODE_DOT: ybar [nk][n_own][N]
  float2* out;          // APPLY / OCC: [nk][n_own][N]
  double* partial;      // ENERGY / DOT: [nk][n_own]
  const double* occ;    // [nk_occ][n_occ] occupations of the occupied orbitals
  const double* occ_own;  // MODE_ENERGY: [nk_own][n_occ] occupations of the owners
  const float* vtab;    // [nq][N] kernel rows v(|G+q|) (or d v / d omega)
  const int* qidx;      // [nk_tgt][nk_occ] row of q = k - k' (k a target point, k' occupied)
  int nk_own, nk_part;  // k-points of the owners / of the partners (the sampled k' when the
                        // owners are targets, all target k-points for MODE_OCC)
  int n_own, n_part, n_occ;
  int ntiles;           // ceil(n_own / slots)
  float scale;          // -alpha / (N_k * N): per-pair scale is scale * f
  int nsplit;           // the k' loop is split into nsplit work items per owner tile
  size_t split_stride;  // elements between the per-split outputs (out: float2, partial: double)
  int* status;          // device status word for failed device-side waits (may be null)
  int inject;           // test hook: 1 = the staged kernel never issues its first partner copy
  int blk;              // pencil-load kernel: own, part and part2 are in the pencil-blocked
                        // layout (OrbBlk below) instead of [x][y][z]; out stays [x][y][z]
  float2* comp;         // APPLY / OCC: running sums s, c of the compensated accumulation: per
                        // owner orbital of each split, s then c in the pencil-blocked layout
                        // (2 OrbBlk::NBK complex), owners in the order of out
  // MODE_OCC with the omega gradient fused in (vtab2 non-null): the rows d v / d omega (scaled
  // like vtab), one FP64 partial per item, and per CTA of the launch one spectrum of each owner
  // slot (T blocked grids, float2) kept from the first chain to the second.
  const float* vtab2;
  double* partial2;
  float2* spec;
  int item0;            // pencil-load launches: items item0 .. item0 + item_count - 1
  int item_count;       // (0: all items)
};

// Work item `item` -> (split, k, tile), split slowest: the items of one k' split (one range of
// partner orbitals) run together, so the partners a wave reads stay in L2 from wave to wave.
struct ItemIdx {
  int split, k, tile;
  __device__ __forceinline__ ItemIdx(const PairArgs& a, int item) {
    const int per_split = a.nk_own * a.ntiles;
    split = item / per_split;
    const int rem = item - split * per_split;
    k = rem / a.ntiles;
    tile = rem - k * a.ntiles;
  }
};

// ---------------------------------------------------------------------------------------
// Compensated accumulation over k' (Sec. II C, Eq. "Fock": V_x u sums the pair terms over
// every k' and every occupied band).  The TMEM accumulator of a pencil holds the sum over the
// bands of a group of consecutive k' (in FP32; fold_span k-points, so that a group holds at
// least 16 band terms where the bands are fewer).  When the group ends it is added to the pencil's running
// sum s with Knuth's TwoSum, whose exact rounding error is added to a second running sum c;
// the pencil's result is s + c, written to the output (or the work item's split partial) by
// the last fold.  s and c live in PairArgs::comp in the pencil-blocked layout (a warp's 32
// pencils move as 512 contiguous bytes per access); only the thread that owns a pencil touches
// its sums.  The dot epilogues (energy, d/d omega) instead add each group's FP32 pencil dot to
// an FP64 sum.
// ---------------------------------------------------------------------------------------

// k-points per fold group: one, or enough for 16 partner bands
__host__ __device__ __forceinline__ int fold_span(int n_part) { return n_part >= 16 ? 1 : (16 + n_part - 1) / n_part; }

// a + b = s + err exactly, s = fl(a + b) (TwoSum; no fast-math reassociation in this build)
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
  const float s = a + b;
  const float bb = s - a;
  err = (a - (s - bb)) + (b - bb);
  return s;
}

__device__ __forceinline__ void fold4(float4& sv, float4& cv, const float4 s0, const float4 c0) {
  float er;
  sv.x = two_sum(s0.x, sv.x, er);
  cv.x = c0.x + er;
  sv.y = two_sum(s0.y, sv.y, er);
  cv.y = c0.y + er;
  sv.z = two_sum(s0.z, sv.z, er);
  cv.z = c0.z + er;
  sv.w = two_sum(s0.w, sv.w, er);
  cv.w = c0.w + er;
}

// Folds one group row g (z-pencil p, 2n floats) into the running sums of its orbital: s at
// sums (n/2 float4 per pencil, pencil-blocked), c at sums + NBK/2 float4.  first: s = g (c is
// not written); second: c is still zero (not read); last: the final s + c goes to out4 (the
// pencil in [x][y][z] order, n/2 float4).  With first and last together out4 = g.
template <int n>
__device__ __forceinline__ void fold_group(const float* g, float4* __restrict__ sums, int p, float4* out4,
                                           bool first, bool second, bool last) {
  float4* s4 = sums + (size_t)(p >> 5) * (n / 2) * 32 + (p & 31);
  float4* c4 = s4 + blocked_stride(n) / 2;
#pragma unroll
  for (int e = 0; e < n / 2; ++e) {
    float4 sv = make_float4(g[4 * e], g[4 * e + 1], g[4 * e + 2], g[4 * e + 3]);
    float4 cv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!first) fold4(sv, cv, s4[32 * e], second ? make_float4(0.f, 0.f, 0.f, 0.f) : c4[32 * e]);
    if (last) {
      out4[e] = make_float4(sv.x + cv.x, sv.y + cv.y, sv.z + cv.z, sv.w + cv.w);
    } else {
      s4[32 * e] = sv;
      if (!first) c4[32 * e] = cv;
    }
  }
}

// fold_group on the float4 chunks e0 .. e0 + count - 1 of the row only (g: their 4 count
// floats), for callers that move the accumulator in pieces.
template <int n>
__device__ __forceinline__ void fold_chunks(const float* g, float4* __restrict__ sums, int p, float4* out4, bool first,
                                            bool second, bool last, int e0, int count) {
  float4* s4 = sums + (size_t)(p >> 5) * (n / 2) * 32 + (p & 31);
  float4* c4 = s4 + blocked_stride(n) / 2;
#pragma unroll
  for (int i = 0; i < count; ++i) {
    const int e = e0 + i;
    float4 sv = make_float4(g[4 * i], g[4 * i + 1], g[4 * i + 2], g[4 * i + 3]);
    float4 cv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!first) fold4(sv, cv, s4[32 * e], second ? make_float4(0.f, 0.f, 0.f, 0.f) : c4[32 * e]);
    if (last) {
      out4[e] = make_float4(sv.x + cv.x, sv.y + cv.y, sv.z + cv.z, sv.w + cv.w);
    } else {
      s4[32 * e] = sv;
      if (!first) c4[32 * e] = cv;
    }
  }
}

// The same fold with the running sums in TMEM (the layouts that have the columns): s at ts
// (2n columns, FP32), c at tc (n columns, bf16 pairs: c is the sum of rounding errors, about
// 1e-7 of s, so its own 2^-9 rounding is far below the FP32 resolution of s).  Warp-wide
// (TMEM); out4: the pencil in [x][y][z] order, written by the last fold, or null (inactive).
template <int n>
__device__ __forceinline__ void fold_group_tmem(const float* g, uint32_t ts, uint32_t tc, float4* out4, bool first,
                                                bool second, bool last) {
  float sv[2 * n], cv[2 * n];
  if (first) {
#pragma unroll
    for (int e = 0; e < 2 * n; ++e) {
      sv[e] = g[e];
      cv[e] = 0.f;
    }
  } else {
    TmemRow<2 * n>::load(ts, sv);
    if (second) {
#pragma unroll
      for (int e = 0; e < 2 * n; ++e) cv[e] = 0.f;
    } else {
      float cp[n];
      TmemRow<n>::load(tc, cp);
#pragma unroll
      for (int e = 0; e < n; ++e) {
        const float2 c2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&cp[e]));
        cv[2 * e] = c2.x;
        cv[2 * e + 1] = c2.y;
      }
    }
#pragma unroll
    for (int e = 0; e < 2 * n; ++e) {
      float er;
      sv[e] = two_sum(sv[e], g[e], er);
      cv[e] += er;
    }
  }
  if (last) {
    if (out4) {
#pragma unroll
      for (int e = 0; e < n / 2; ++e)
        out4[e] = make_float4(sv[4 * e] + cv[4 * e], sv[4 * e + 1] + cv[4 * e + 1], sv[4 * e + 2] + cv[4 * e + 2],
                              sv[4 * e + 3] + cv[4 * e + 3]);
    }
  } else {
    TmemRow<2 * n>::store(ts, sv);
    float cp[n];
#pragma unroll
    for (int e = 0; e < n; ++e) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(cv[2 * e], cv[2 * e + 1]);
      cp[e] = *reinterpret_cast<const float*>(&h);
    }
    TmemRow<n>::store(tc, cp);
  }
}

// running sums of owner orbital `orb` (counted in the order of out, splits included)
__device__ __forceinline__ float4* sums_of(const PairArgs& a, size_t orb, size_t nbk) {
  return reinterpret_cast<float4*>(a.comp + orb * 2 * nbk);
}

// Re <w | g> over one pencil (n complex values; g interleaved), FP32
template <int n>
__device__ __forceinline__ float pencil_dot(const cpx<float> (&w)[n], const float* g) {
  float d = 0.f;
#pragma unroll
  for (int e = 0; e < n; ++e) d = fmaf(w[e].x, g[2 * e], fmaf(w[e].y, g[2 * e + 1], d));
  return d;
}

// L1 policy of the 16-byte chunks of a pencil-blocked orbital (a warp reads 512 contiguous
// bytes per access) in the one-pencil-per-thread layout, whose 96-register budget spills a few
// loop-invariant values to local memory: those reloads must hit L1.  The partner is read twice
// per pair, in the Z forward and the Z inverse stage, so its first read stays in L1 longest
// (evict_last); the owner and the partner's last read are plain loads.  Streaming those two past
// L1 (L1::no_allocate or L1::evict_first) also marks their lines evict-first in L2, where the
// owner, re-read by every pair of its target, must stay: on the 24^3, 3x3x3 k, 8-band cell it
// raised DRAM reads from 60 MB to 2.76 GB a launch (L2 hit rate 95% -> 64%) and the 24^3,
// 8x8x8 k, 16 + 16-band apply from 7.32 s to 7.97 s.  An explicit L2::evict_normal or
// evict_last cache hint on the streamed loads keeps L2 but costs 25% of the time (its policy
// register and extra instructions).  The layouts with two pencils a thread (no spills) use
// plain loads throughout.
enum LdPolicy : int { LD_NORMAL = 0, LD_KEEP = 1 };
constexpr int kLdOwner = LD_NORMAL;
constexpr int kLdPartnerFirst = LD_KEEP;
constexpr int kLdPartnerLast = LD_NORMAL;

template <int POL>
__device__ __forceinline__ float4 ldg_pol(const float4* p) {
  float4 v;
  if constexpr (POL == LD_KEEP) {
    asm volatile("ld.global.nc.L1::evict_last.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
  } else {
    v = __ldg(p);
  }
  return v;
}

template <int n>
__device__ __forceinline__ void load_pencil_global(cpx<float> (&v)[n], const float2* __restrict__ p) {
  const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int e = 0; e < n / 2; ++e) {
    const float4 w = __ldg(p4 + e);
    v[2 * e] = {w.x, w.y};
    v[2 * e + 1] = {w.z, w.w};
  }
}

// Pencil-blocked orbital layout, read by the pencil-load kernel.  A thread of that kernel reads
// its own z-pencil (n complex, 8n bytes); in the natural layout the 32 lanes of a warp are 8n
// bytes apart, so every 16-byte access of the warp touches 32 cache lines.  Blocked, the
// z-pencils p = 32 b + l (l < 32) of block b store their elements (2e, 2e + 1) as 16-byte chunks
// side by side: chunk (b, e, l) at float4 index (b n/2 + e) 32 + l.  A warp reading 32
// consecutive pencils then reads 512 contiguous bytes per access.  NBK: complex per blocked
// orbital (the last block is padded to 32 pencils).
template <int n>
struct OrbBlk {
  static constexpr size_t NBK = blocked_stride(n);
};

// Z-pencil p (= x n + y) of one orbital, natural (blk = 0) or pencil-blocked (blk = 1).
template <int n, int POL = LD_NORMAL>
__device__ __forceinline__ void load_pencil(cpx<float> (&v)[n], const float2* __restrict__ orb, int p, int blk) {
  if (blk) {
    const float4* b4 = reinterpret_cast<const float4*>(orb) + (size_t)(p >> 5) * (n / 2) * 32 + (p & 31);
#pragma unroll
    for (int e = 0; e < n / 2; ++e) {
      const float4 w = ldg_pol<POL>(b4 + 32 * e);
      v[2 * e] = {w.x, w.y};
      v[2 * e + 1] = {w.z, w.w};
    }
  } else {
    load_pencil_global<n>(v, orb + (size_t)p * n);
  }
}

// complex elements between consecutive orbitals of an array in the given layout
template <int n>
__host__ __device__ __forceinline__ size_t orb_stride(int blk) {
  return blk ? (size_t)OrbBlk<n>::NBK : (size_t)n * n * n;
}

// One pencil of the smem grid: n complex values at base + e * stride.  A stride of 1 with
// VEC = 2 moves two neighbours per 128-bit access.
template <int n, int VEC>
__device__ __forceinline__ void load_s(cpx<float> (&v)[n], const float2* g, int base, int stride) {
  if constexpr (VEC == 2) {
#pragma unroll
    for (int e = 0; e < n / 2; ++e) {
      const float4 w = *reinterpret_cast<const float4*>(g + base + 2 * e);
      v[2 * e] = {w.x, w.y};
      v[2 * e + 1] = {w.z, w.w};
    }
  } else {
#pragma unroll
    for (int e = 0; e < n; ++e) {
      const float2 w = g[base + e * stride];
      v[e] = {w.x, w.y};
    }
  }
}

template <int n, int VEC>
__device__ __forceinline__ void store_s(const cpx<float> (&v)[n], float2* g, int base, int stride) {
  if constexpr (VEC == 2) {
#pragma unroll
    for (int e = 0; e < n / 2; ++e)
      *reinterpret_cast<float4*>(g + base + 2 * e) = make_float4(v[2 * e].x, v[2 * e].y, v[2 * e + 1].x, v[2 * e + 1].y);
  } else {
#pragma unroll
    for (int e = 0; e < n; ++e) g[base + e * stride] = make_float2(v[e].x, v[e].y);
  }
}

// Pencil p (0 <= p < n^2) of each stage; lanes of a warp take consecutive p.
template <int n>
struct Pencil {
  using G = Geo<n>;
  int zs;      // Z stage: smem base of z-pencil (x, y), stride 1
  int zg;      // Z stage: global offset (x n + y) n of that pencil
  int ys;      // Y stage: pencil (x = p / n, z = p % n), stride P
  int xs;      // X stage: pencil (y = p / n, z = p % n), stride Q
  int vr;      // X stage: kernel row element (x, y, z) at x n^2 + p
  __host__ __device__ __forceinline__ explicit Pencil(int p) {
    const int hi = p / n, lo = p - hi * n;
    const int zx = G::ZFAST_Y ? hi : lo;
    const int zy = G::ZFAST_Y ? lo : hi;
    zs = zx * G::Q + zy * G::P;
    zg = (zx * n + zy) * n;
    ys = hi * G::Q + lo;
    xs = hi * G::P + lo;
    vr = p;
  }
};

// Stage Y (DIR) for the PPT pencils of the thread (pencil t + ps NN/PPT): load, FFT, store.
template <int n, int DIR, int PPT = 2, int TS = Geo<n>::NN / PPT>
__device__ __forceinline__ void stage_y(float2* g, int t, bool valid) {
  using G = Geo<n>;
#pragma unroll 1
  for (int ps = 0; ps < PPT; ++ps) {
    if (TS * PPT != G::NN && t + ps * TS >= G::NN) break;  // whole warps past the last pencil
    const Pencil<n> pc(t + ps * TS);
    cpx<float> v[n];
    load_s<n, 1>(v, g, pc.ys, G::P);
    fft<n, DIR, float>(v);
    if (valid) store_s<n, 1>(v, g, pc.ys, G::P);
  }
}

// X-stage pencil of thread t when each thread owns one X pencil: the first R of the n^2
// pencils (y, z), p = y n + z, grouped 16 to a half-warp with distinct 8-byte banks
// (y P + z mod 16) as long as every bank class still has a member, the rest of those R after
// them; pencils R and up keep their place.  With the pitch P = n the identity already has
// this property; with P != n (20^3: P = 21) consecutive pencils wrap from one y row to the
// next inside a half-warp and two of them share a bank.
template <int n>
struct XPermTable {
  unsigned short v[n * n];
};
template <int n, int R>
constexpr XPermTable<n> make_xperm() {
  constexpr int NN = n * n, P = Geo<n>::P;
  XPermTable<n> t{};
  unsigned short bucket[16][NN / 16 + 16] = {};
  int cnt[16] = {};
  for (int p = 0; p < R; ++p) {
    const int r = ((p / n) * P + p % n) % 16;
    bucket[r][cnt[r]++] = (unsigned short)p;
  }
  int ming = NN;
  for (int r = 0; r < 16; ++r) ming = cnt[r] < ming ? cnt[r] : ming;
  int k = 0;
  for (int g = 0; g < ming; ++g)
    for (int r = 0; r < 16; ++r) t.v[k++] = bucket[r][g];
  for (int r = 0; r < 16; ++r)
    for (int g = ming; g < cnt[r]; ++g) t.v[k++] = bucket[r][g];
  for (int p = R; p < NN; ++p) t.v[k++] = (unsigned short)p;
  return t;
}
template <int n, int R>
__device__ const XPermTable<n> kXPerm = make_xperm<n, R>();

template <int n, bool XP, int R = n * n>
__device__ __forceinline__ int x_pencil(int p) {
  if constexpr (XP && Geo<n>::P != n) {
    return kXPerm<n, R>.v[p];
  } else {
    return p;
  }
}

// Stage X: FFT, multiply by the kernel row (cached in TMEM, already times -alpha/(N_k N))
// times the occupation f, inverse FFT, for the PPT pencils.  Warp-wide (TMEM loads).
// XP: the bank-spread X-pencil order of x_pencil over the first XR.  xs_tab (one pencil per
// thread): each thread's X pencil as its smem offset, in that order, from a table in shared
// memory; its kernel row then comes in eight TMEM columns at a time after the forward
// transform instead of being held through it (fewer live registers).
template <int n, int PPT = 2, bool XP = false, int XR = n * n, int TS = Geo<n>::NN / PPT>
__device__ __forceinline__ void stage_x(float2* g, int t, bool valid, uint32_t ttab, float f,
                                        const unsigned short* xs_tab = nullptr) {
  using G = Geo<n>;
#pragma unroll 1
  for (int ps = 0; ps < PPT; ++ps) {
    if (TS * PPT != G::NN && t + ps * TS >= G::NN) break;
    cpx<float> v[n];
    if (PPT == 1 && n % 8 == 0 && xs_tab != nullptr) {
      const int xs = xs_tab[t];
      load_s<n, 1>(v, g, xs, G::Q);
      fft<n, -1, float>(v);
#pragma unroll
      for (int c = 0; c < n / 8; ++c) {
        float tv[8];
        tmem_ld8(ttab + (uint32_t)(8 * c), tv);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float w = tv[e] * f;
          v[8 * c + e].x *= w;
          v[8 * c + e].y *= w;
        }
      }
      fft<n, +1, float>(v);
      if (valid) store_s<n, 1>(v, g, xs, G::Q);
    } else {
      const Pencil<n> pc(x_pencil<n, XP, XR>(t + ps * TS));
      float tv[n];
      TmemRow<n>::load(ttab + (uint32_t)(ps * n), tv);
      load_s<n, 1>(v, g, pc.xs, G::Q);
      fft<n, -1, float>(v);
#pragma unroll
      for (int e = 0; e < n; ++e) {
        const float w = tv[e] * f;
        v[e].x *= w;
        v[e].y *= w;
      }
      fft<n, +1, float>(v);
      if (valid) store_s<n, 1>(v, g, pc.xs, G::Q);
    }
  }
}

// Stage X of the two chains of MODE_OCC with the omega gradient fused in (Sec. II C, the
// derivative of Eq. "Fock" with respect to omega).  With A = F(conj(u_j) u_i) and
// B = F(conj(u_j) ybar_i) the unnormalised spectra the first and second chain reach here,
//   Re sum_r conj(ybar_i) u_j K'_q(conj(u_j) u_i) (scaled by -alpha f / (N_k N))
//     = Re sum_G dvs(G) f A(G) conj(B(G))   (Parseval; dvs = d v / d omega * scale),
// the term the separate omega pass computes in real space.  SPEC = 1 (first chain) stores A
// per X pencil in the pencil-blocked layout at spec; SPEC = 2 (second chain) reads it back and
// adds the sum to dsum.  Otherwise as stage_x.
template <int n, int SPEC, int PPT = 2, int TS = Geo<n>::NN / PPT>
__device__ __forceinline__ void stage_x_occ(float2* g, int t, bool valid, uint32_t ttab, float f, float2* spec,
                                            const float* __restrict__ dvrow, float dscale, double& dsum) {
  using G = Geo<n>;
#pragma unroll 1
  for (int ps = 0; ps < PPT; ++ps) {
    if (TS * PPT != G::NN && t + ps * TS >= G::NN) break;
    const int p = t + ps * TS;
    const Pencil<n> pc(p);
    float tv[n];
    TmemRow<n>::load(ttab + (uint32_t)(ps * n), tv);
    cpx<float> v[n];
    load_s<n, 1>(v, g, pc.xs, G::Q);
    fft<n, -1, float>(v);
    float4* s4 = reinterpret_cast<float4*>(spec) + (size_t)(p >> 5) * (n / 2) * 32 + (p & 31);
    if constexpr (SPEC == 1) {
      if (valid) {
#pragma unroll
        for (int e = 0; e < n / 2; ++e) s4[32 * e] = make_float4(v[2 * e].x, v[2 * e].y, v[2 * e + 1].x, v[2 * e + 1].y);
      }
    } else {
      float d = 0.f;
#pragma unroll
      for (int e = 0; e < n / 2; ++e) {
        const float4 a = s4[32 * e];
        const float w0 = __ldg(dvrow + (2 * e) * G::NN + p), w1 = __ldg(dvrow + (2 * e + 1) * G::NN + p);
        d = fmaf(w0, fmaf(a.x, v[2 * e].x, a.y * v[2 * e].y), d);
        d = fmaf(w1, fmaf(a.z, v[2 * e + 1].x, a.w * v[2 * e + 1].y), d);
      }
      if (valid) dsum += (double)d * (double)(dscale * f);
    }
#pragma unroll
    for (int e = 0; e < n; ++e) {
      const float w = tv[e] * f;
      v[e].x *= w;
      v[e].y *= w;
    }
    fft<n, +1, float>(v);
    if (valid) store_s<n, 1>(v, g, pc.xs, G::Q);
  }
}

// Kernel row v(|G+q|) * scale of this thread's PPT X-pencils into the TMEM cache.
template <int n, int PPT = 2, bool XP = false, int XR = n * n, int TS = Geo<n>::NN / PPT>
__device__ __forceinline__ void cache_kernel_row(int t, uint32_t ttab, const float* __restrict__ vrow, float scale) {
  using G = Geo<n>;
#pragma unroll 1
  for (int ps = 0; ps < PPT; ++ps) {
    if (TS * PPT != G::NN && t + ps * TS >= G::NN) break;
    const int p = x_pencil<n, XP, XR>(t + ps * TS);
    float tv[n];
#pragma unroll
    for (int e = 0; e < n; ++e) tv[e] = __ldg(vrow + e * G::NN + p) * scale;
    TmemRow<n>::store(ttab + (uint32_t)(ps * n), tv);
  }
}

// Z forward for the thread's pencils: v = conj(a) * b, FFT along z, store.
// a, b: orbitals in layout blk.
template <int n, int PPT = 2, int TS = Geo<n>::NN / PPT>
__device__ __forceinline__ void stage_z_forward(float2* g, int t, bool valid, const float2* __restrict__ a,
                                                const float2* __restrict__ b, int blk) {
  using G = Geo<n>;
  static_assert(G::ZFAST_Y == 1, "z-pencil p of the Z stage is (x, y) = (p / n, p % n)");
#pragma unroll 1
  for (int ps = 0; ps < PPT; ++ps) {
    if (TS * PPT != G::NN && t + ps * TS >= G::NN) break;
    const int p = t + ps * TS;
    const Pencil<n> pc(p);
    cpx<float> v[n];
    if constexpr (PPT == 1) {
      // one pencil per thread (many warps, few registers each): the two orbitals' 16-byte
      // chunks are read and multiplied one pair at a time, so that only one pencil is live
      const int off = blk ? (p >> 5) * (n / 2) * 32 + (p & 31) : p * (n / 2);
      const float4* a4 = reinterpret_cast<const float4*>(a) + off;
      const float4* b4 = reinterpret_cast<const float4*>(b) + off;
#pragma unroll
      for (int e = 0; e < n / 2; ++e) {
        const float4 w = blk ? ldg_pol<kLdPartnerFirst>(a4 + 32 * e) : __ldg(a4 + e);
        const float4 u = blk ? ldg_pol<kLdOwner>(b4 + 32 * e) : __ldg(b4 + e);
        v[2 * e] = {w.x * u.x + w.y * u.y, w.x * u.y - w.y * u.x};
        v[2 * e + 1] = {w.z * u.z + w.w * u.w, w.z * u.w - w.w * u.z};
      }
    } else {
      cpx<float> w[n];
      load_pencil<n>(w, a, p, blk);
      load_pencil<n>(v, b, p, blk);
#pragma unroll
      for (int e = 0; e < n; ++e) v[e] = {w[e].x * v[e].x + w[e].y * v[e].y, w[e].x * v[e].y - w[e].y * v[e].x};
    }
    fft<n, -1, float>(v);
    if (valid) store_s<n, G::ZVEC>(v, g, pc.zs, 1);
  }
}

enum Epi : int {
  EPI_MUL = 0,      // acc += w * phi
  EPI_CONJPHI = 1,  // acc += conj(phi) * w
  EPI_WCONJ = 2,    // acc += w * conj(phi)
};

// One complex term of the Z-inverse epilogue into the accumulator (ar, ai).
template <int EPI>
__device__ __forceinline__ void epilogue_mac(float& ar, float& ai, const cpx<float> w, const cpx<float> v) {
  if constexpr (EPI == EPI_MUL) {  // acc += w phi
    ar = fmaf(w.x, v.x, fmaf(-w.y, v.y, ar));
    ai = fmaf(w.x, v.y, fmaf(w.y, v.x, ai));
  } else if constexpr (EPI == EPI_CONJPHI) {  // acc += conj(phi) w
    ar = fmaf(v.x, w.x, fmaf(v.y, w.y, ar));
    ai = fmaf(v.x, w.y, fmaf(-v.y, w.x, ai));
  } else {  // acc += w conj(phi)
    ar = fmaf(w.x, v.x, fmaf(w.y, v.y, ar));
    ai = fmaf(w.y, v.x, fmaf(-w.x, v.y, ai));
  }
}

// Z inverse for the thread's pencils, then the epilogue into each pencil's TMEM row.
// Executed by every thread of the warp (TMEM accesses are warp-wide).
template <int n, int EPI, int PPT = 2, int TS = Geo<n>::NN / PPT>
__device__ __forceinline__ void stage_z_inverse(const float2* g, int t, const float2* __restrict__ wbase,
                                                uint32_t trow0, int blk) {
  using G = Geo<n>;
#pragma unroll 1
  for (int ps = 0; ps < PPT; ++ps) {
    if (TS * PPT != G::NN && t + ps * TS >= G::NN) break;
    const int p = t + ps * TS;
    const Pencil<n> pc(p);
    cpx<float> v[n];
    load_s<n, G::ZVEC>(v, g, pc.zs, 1);
    fft<n, +1, float>(v);
    const uint32_t trow = trow0 + (uint32_t)(ps * G::ROW);
    if constexpr (PPT == 1 && n % 4 == 0) {
      // one pencil per thread: the accumulator row and the partner move four complex values
      // (eight TMEM columns, two 16-byte chunks) at a time, so that only phi stays live
      const int off = blk ? (p >> 5) * (n / 2) * 32 + (p & 31) : p * (n / 2);
      const float4* w4 = reinterpret_cast<const float4*>(wbase) + off;
#pragma unroll
      for (int c = 0; c < n / 4; ++c) {
        float acc[8];
        tmem_ld8(trow + (uint32_t)(8 * c), acc);
        const float4 w0 = blk ? ldg_pol<kLdPartnerLast>(w4 + 32 * (2 * c)) : __ldg(w4 + 2 * c);
        const float4 w1 = blk ? ldg_pol<kLdPartnerLast>(w4 + 32 * (2 * c + 1)) : __ldg(w4 + 2 * c + 1);
        const cpx<float> w[4] = {{w0.x, w0.y}, {w0.z, w0.w}, {w1.x, w1.y}, {w1.z, w1.w}};
#pragma unroll
        for (int q = 0; q < 4; ++q) epilogue_mac<EPI>(acc[2 * q], acc[2 * q + 1], w[q], v[4 * c + q]);
        tmem_st8(trow + (uint32_t)(8 * c), acc);
      }
    } else {
      float acc[G::ROW];
      TmemRow<G::ROW>::load(trow, acc);
      cpx<float> w[n];
      load_pencil<n>(w, wbase, p, blk);
#pragma unroll
      for (int e = 0; e < n; ++e) epilogue_mac<EPI>(acc[2 * e], acc[2 * e + 1], w[e], v[e]);
      TmemRow<G::ROW>::store(trow, acc);
    }
  }
}

// Threads per x-slab barrier of the one-pencil layout, else 0.  With one pencil per thread
// and T = 1, thread p holds the Z pencil (x, y) = (p / n, p % n) and the Y pencil
// (x, z) = (p / n, p % n): the Z and Y stages of a pair touch only the x-planes of their own
// threads, and only the X stage reads across x.  The barriers Z forward -> Y forward and
// Y inverse -> Z inverse then need only the threads of the same x-planes: lcm(n, 32) threads
// (whole warps, n^2 / lcm(n, 32) groups, named barriers 1 ...).  The groups run ahead of one
// another between the two CTA-wide barriers around the X stage, so their shared-memory and
// global-load phases spread out.
constexpr int gcd_int(int a, int b) { return b == 0 ? a : gcd_int(b, a % b); }
template <int n, int PPT, int TS>
constexpr int slab_bar_threads() {
  constexpr int L = n / gcd_int(n, 32) * 32;
  if constexpr (PPT == 1 && TS == Geo<n>::NN && Geo<n>::T == 1 && Geo<n>::ZFAST_Y == 1 && Geo<n>::NN % L == 0 &&
                Geo<n>::NN / L <= 15 && Geo<n>::NN / L > 1) {
    return L;
  } else {
    return 0;
  }
}

// Barrier of the x-slab of thread tid (SB threads; named barrier 1 + tid / SB), or of the CTA.
template <int SB>
__device__ __forceinline__ void slab_sync() {
  if constexpr (SB > 0) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)threadIdx.x / SB), "n"(SB) : "memory");
  } else {
    __syncthreads();
  }
}

// One pair chain between the Z stages; all threads of the CTA call it together.  xs_tab (one
// pencil per thread): the smem offset of each thread's X pencil in the bank-spread order.
template <int n, int PPT = 2, int TS = Geo<n>::NN / PPT>
__device__ __forceinline__ void pair_middle(float2* g, int t, bool valid, uint32_t ttab, float f, bool warp_on = true,
                                            const unsigned short* xs_tab = nullptr) {
  constexpr int SB = slab_bar_threads<n, PPT, TS>();
  slab_sync<SB>();
  if (warp_on) stage_y<n, -1, PPT, TS>(g, t, valid);
  __syncthreads();
  if (warp_on) stage_x<n, PPT, false, n * n, TS>(g, t, valid, ttab, f, xs_tab);
  __syncthreads();
  if (warp_on) stage_y<n, +1, PPT, TS>(g, t, valid);
  slab_sync<SB>();
}

}  // namespace hse

// the tensor-core Y and X stages (pair_middle_tc), which use the definitions above
#include "pairconv_tc.cuh"

namespace hse {

// The same with stage_x_occ (MODE_OCC with the omega gradient fused in).
template <int n, int SPEC, int PPT = 2, int TS = Geo<n>::NN / PPT>
__device__ __forceinline__ void pair_middle_occ(float2* g, int t, bool valid, uint32_t ttab, float f, float2* spec,
                                                const float* dvrow, float dscale, double& dsum, bool warp_on) {
  __syncthreads();
  if (warp_on) stage_y<n, -1, PPT, TS>(g, t, valid);
  __syncthreads();
  if (warp_on) stage_x_occ<n, SPEC, PPT, TS>(g, t, valid, ttab, f, spec, dvrow, dscale, dsum);
  __syncthreads();
  if (warp_on) stage_y<n, +1, PPT, TS>(g, t, valid);
  __syncthreads();
}

// One work item `item` = (split, k, tile) of a launch.  The CTA may have more threads than
// the item needs (the batched kernel runs every grid side in one block shape): warps with
// warp_on == false skip all work and TMEM traffic but pass every barrier.  tbase: the CTA's
// TMEM allocation, at least Geo<n>::TMEM_COLS columns for this block's warp count.
// spec: this CTA's spectrum scratch (T blocked grids) when args.vtab2 is set (MODE_OCC).
// TC: the Y and X stages on the tensor cores (stage_y_tc / stage_x_tc; the DFT tables follow
// the grids in shared memory), for the modes with owner = target.
// BLK: the orbital layout args.blk as a compile-time constant (0 or 1; -1: read at run time).
template <int n, int MODE, int PPT = 2, int TSX = Geo<n>::NN / PPT, bool TC = false, int BLK = -1>
__device__ __forceinline__ void pairconv_item(const PairArgs& args, int item, float4* smem4, uint32_t tbase,
                                              bool warp_on, float2* spec = nullptr) {
  using G = Geo<n>;
  using GP = GeoP<n, PPT, TSX>;
  constexpr int TS = GP::TS;
  static_assert(!TC || MODE != MODE_OCC, "the tensor-core stages serve the owner = target modes");

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  // every kernel that runs an item launches GP::THREADS threads: where those are exactly the
  // T * TS pencil threads every thread is valid, which the compiler then knows (uniform owner,
  // band and occupation values, fewer vector registers)
  const bool valid = (GP::THREADS == G::T * TS) || tid < G::T * TS;
  const int slot = valid ? tid / TS : 0;
  const int t = valid ? tid - slot * TS : 0;
  float2* g = reinterpret_cast<float2*>(smem4) + slot * G::GRID_CPX;

  // tensor memory for the accumulators: warp w uses lanes 32 (w % 4) .. +31, columns from
  // (w / 4) * COLS_PER_WARP; the thread's pencil pass ps is the row at + ps * ROW.
  const uint32_t trow0 = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * GP::COLS_PER_WARP);
  const uint32_t ttab = trow0 + (uint32_t)GP::TAB;

  // work item: (split, k, tile); split s covers partner k-points
  // [s nk_part / nsplit, (s+1) nk_part / nsplit)
  const ItemIdx it(args, item);
  const int split = it.split;
  const int k = it.k;
  const int band = it.tile * G::T + slot;
  const int kp_begin = (int)(((long long)split * args.nk_part) / args.nsplit);
  const int kp_end = (int)(((long long)(split + 1) * args.nk_part) / args.nsplit);
  const bool active = valid && band < args.n_own;
  const int bandc = active ? band : 0;
  const int blk = BLK >= 0 ? BLK : args.blk;
  const size_t ostr = orb_stride<n>(blk);
  const float2* own = args.own + ((size_t)k * args.n_own + bandc) * ostr;

  if (warp_on) {
    float z[G::ROW];
#pragma unroll
    for (int e = 0; e < G::ROW; ++e) z[e] = 0.f;
#pragma unroll
    for (int ps = 0; ps < PPT; ++ps) TmemRow<G::ROW>::store(trow0 + (uint32_t)(ps * G::ROW), z);
  }
  // the bank-spread X-pencil order (x_pencil) of the one-pencil layout, as smem offsets of
  // each thread's X pencil in a table in shared memory (read once per pair, no global lookup)
  constexpr bool kXTab = PPT == 1 && n % 8 == 0 && !TC && MODE != MODE_OCC && G::T == 1 && G::P != n;
  __shared__ unsigned short xs_tab[kXTab ? G::NN : 1];
  if constexpr (kXTab) {
    for (int i = tid; i < G::NN; i += blockDim.x) xs_tab[i] = (unsigned short)Pencil<n>(x_pencil<n, true>(i)).xs;
    // ordered before its first use by the CTA barrier in front of the first X stage
  }

  // compensated accumulation over the k' groups (one group per k'): APPLY / OCC keep the
  // running sums in the item's output region ([x][y][z]) and in args.comp; ENERGY / DOT add
  // group dots to dsum (FP64)
  const size_t oofs = split * args.split_stride + ((size_t)k * args.n_own + bandc) * G::N;
  float4* sums = (MODE == MODE_APPLY || MODE == MODE_OCC) ? sums_of(args, oofs / G::N, OrbBlk<n>::NBK) : nullptr;
  const float2* lhs = (MODE == MODE_DOT) ? args.part2 + ((size_t)k * args.n_own + bandc) * ostr : own;
  double dsum = 0.0;
  auto fold = [&](bool first, bool second, bool last) {
    if (!warp_on) return;
#pragma unroll 1
    for (int ps = 0; ps < PPT; ++ps) {
      if (TS * PPT != G::NN && t + ps * TS >= G::NN) break;
      const uint32_t trow = trow0 + (uint32_t)(ps * G::ROW);
      const int p = t + ps * TS;
      if constexpr (PPT == 1 && n % 4 == 0) {
        // one pencil per thread: eight accumulator columns (two 16-byte chunks) at a time
        const int loff = blk ? (p >> 5) * (n / 2) * 32 + (p & 31) : p * (n / 2);
        float dpart = 0.f;
#pragma unroll
        for (int c = 0; c < n / 4; ++c) {
          float acc[8];
          tmem_ld8(trow + (uint32_t)(8 * c), acc);
          if constexpr (MODE == MODE_APPLY || MODE == MODE_OCC) {
            if (active)
              fold_chunks<n>(acc, sums, p, reinterpret_cast<float4*>(args.out + oofs + (size_t)p * n), first, second,
                             last, 2 * c, 2);
          } else {
            const float4* l4 = reinterpret_cast<const float4*>(lhs) + loff;
            const float4 w0 = blk ? ldg_pol<kLdOwner>(l4 + 32 * (2 * c)) : __ldg(l4 + 2 * c);
            const float4 w1 = blk ? ldg_pol<kLdOwner>(l4 + 32 * (2 * c + 1)) : __ldg(l4 + 2 * c + 1);
            dpart = fmaf(w0.x, acc[0], fmaf(w0.y, acc[1], dpart));
            dpart = fmaf(w0.z, acc[2], fmaf(w0.w, acc[3], dpart));
            dpart = fmaf(w1.x, acc[4], fmaf(w1.y, acc[5], dpart));
            dpart = fmaf(w1.z, acc[6], fmaf(w1.w, acc[7], dpart));
          }
          if (!last) {
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[e] = 0.f;
            tmem_st8(trow + (uint32_t)(8 * c), acc);
          }
        }
        if constexpr (MODE == MODE_ENERGY || MODE == MODE_DOT) dsum += (double)dpart;
      } else {
        float acc[G::ROW];
        TmemRow<G::ROW>::load(trow, acc);
        if constexpr (MODE == MODE_APPLY || MODE == MODE_OCC) {
          if (active)
            fold_group<n>(acc, sums, p, reinterpret_cast<float4*>(args.out + oofs + (size_t)p * n), first, second, last);
        } else {
          cpx<float> w[n];
          load_pencil<n>(w, lhs, p, blk);
          dsum += (double)pencil_dot<n>(w, acc);
        }
        if (!last) {
#pragma unroll
          for (int e = 0; e < G::ROW; ++e) acc[e] = 0.f;
          TmemRow<G::ROW>::store(trow, acc);
        }
      }
    }
  };
  if (kp_begin == kp_end) fold(true, false, true);  // an empty k' range: zeros
  const int fspan = fold_span(args.n_part);

  // MODE_OCC with the omega gradient fused in: this slot's spectrum scratch and FP64 sum
  const bool fuse_w = MODE == MODE_OCC && args.vtab2 != nullptr && spec != nullptr;
  float2* spec_slot = fuse_w ? spec + (size_t)slot * OrbBlk<n>::NBK : nullptr;
  double wsum = 0.0;

  for (int kp = kp_begin; kp < kp_end; ++kp) {
    // q = k_i - k_j: APPLY-like modes own i (at k) and pair with j at kp; OCC owns j (at k)
    const int qrow = (MODE == MODE_OCC) ? args.qidx[kp * args.nk_own + k] : args.qidx[k * args.nk_part + kp];
    const float* dvrow = fuse_w ? args.vtab2 + (size_t)qrow * G::N : nullptr;
    if (warp_on && !TC) {
      if constexpr (kXTab)
        cache_kernel_row<n, PPT, true, n * n, TS>(t, ttab, args.vtab + (size_t)qrow * G::N, args.scale);
      else
        cache_kernel_row<n, PPT, false, n * n, TS>(t, ttab, args.vtab + (size_t)qrow * G::N, args.scale);
    }
    for (int j = 0; j < args.n_part; ++j) {
      const float2* part = args.part + ((size_t)kp * args.n_part + j) * ostr;
      if constexpr (MODE != MODE_OCC) {
        const float f = (float)args.occ[kp * args.n_occ + j];
        if (f == 0.f) continue;  // uniform over the CTA
        if (warp_on) stage_z_forward<n, PPT, TS>(g, t, valid, part, own, blk);          // conj(u_j) u_i
        if constexpr (TC) {
          const TcTables<n>* tct =
              reinterpret_cast<const TcTables<n>*>(reinterpret_cast<const char*>(smem4) + G::SMEM_BYTES);
          pair_middle_tc<n, PPT, TS>(g, t, tct, args.vtab + (size_t)qrow * G::N, args.scale * f, warp_on);
        } else {
          pair_middle<n, PPT, TS>(g, t, valid, ttab, f, warp_on, kXTab ? xs_tab : nullptr);
        }
        if (warp_on) stage_z_inverse<n, EPI_MUL, PPT, TS>(g, t, part, trow0, blk);      // acc += u_j phi
      } else {
        const float f = (float)args.occ[k * args.n_occ + bandc];
        const float2* ybar = args.part2 + ((size_t)kp * args.n_part + j) * ostr;
        // chain 1: rho = conj(u_j) u_i -> phi;  acc += conj(phi) ybar_i
        if (warp_on) stage_z_forward<n, PPT, TS>(g, t, valid, own, part, blk);
        if (fuse_w)
          pair_middle_occ<n, 1, PPT, TS>(g, t, valid, ttab, f, spec_slot, dvrow, args.scale, wsum, warp_on);
        else
          pair_middle<n, PPT, TS>(g, t, valid, ttab, f, warp_on);
        if (warp_on) stage_z_inverse<n, EPI_CONJPHI, PPT, TS>(g, t, ybar, trow0, blk);
        // chain 2: sigma = conj(u_j) ybar_i -> psibar;  acc += u_i conj(psibar)
        if (warp_on) stage_z_forward<n, PPT, TS>(g, t, valid, own, ybar, blk);
        if (fuse_w)
          pair_middle_occ<n, 2, PPT, TS>(g, t, valid, ttab, f, spec_slot, dvrow, args.scale, wsum, warp_on);
        else
          pair_middle<n, PPT, TS>(g, t, valid, ttab, f, warp_on);
        if (warp_on) stage_z_inverse<n, EPI_WCONJ, PPT, TS>(g, t, part, trow0, blk);
      }
    }
    // the end of a fold group (fold_span k-points) or of the item's k' range
    const int grp = (kp - kp_begin) / fspan;
    if (kp == kp_end - 1 || (kp - kp_begin + 1) % fspan == 0) fold(grp == 0, grp == 1, kp == kp_end - 1);
  }

  if constexpr (MODE == MODE_OCC) {
    if (fuse_w) {  // the item's share of d/d omega, one FP64 partial
      __syncthreads();  // the grid buffers are free now; reuse them for the per-thread sums
      double* red = reinterpret_cast<double*>(smem4);
      red[tid] = (active && warp_on) ? wsum : 0.0;  // slots past the last band repeat band 0
      __syncthreads();
      if (tid == 0) {
        double sum = 0.0;
        for (int e = 0; e < (int)blockDim.x; ++e) sum += red[e];
        args.partial2[item] = sum;
      }
      __syncthreads();
    }
  }

  if constexpr (MODE == MODE_ENERGY || MODE == MODE_DOT) {
    // FP64 sum of the group dots with u_i (ENERGY) or ybar_i (DOT), per owner
    const double d = dsum;
    __syncthreads();  // the grid buffers are free now; reuse them for the per-thread partials
    double* red = reinterpret_cast<double*>(smem4);
    red[tid] = (valid && warp_on) ? d : 0.0;
    __syncthreads();
    if (valid && t == 0 && active) {
      double sum = 0.0;
      for (int e = 0; e < TS; ++e) sum += red[slot * TS + e];
      if (MODE == MODE_ENERGY) sum *= args.occ_own[k * args.n_occ + band];
      args.partial[split * args.split_stride + (size_t)k * args.n_own + band] = sum;
    }
  }
}

// BLK: args.blk as a compile-time constant (0 or 1), or -1 (read at run time).
template <int n, int MODE, int MINB, int PPT = 2, int TSX = Geo<n>::NN / PPT, bool TC = false, int BLK = -1>
__global__ void __launch_bounds__(GeoP<n, PPT, TSX>::THREADS, MINB) pairconv_c64_kernel(const PairArgs args) {
  using G = GeoP<n, PPT, TSX>;
  extern __shared__ __align__(16) float4 smem4[];
  __shared__ uint32_t tmem_base_sh;
  const int warp = threadIdx.x >> 5;
  if constexpr (TC)  // the DFT tables after the grids; the barrier below orders them
    tc_build_tables<n>(reinterpret_cast<TcTables<n>*>(reinterpret_cast<char*>(smem4) + Geo<n>::SMEM_BYTES));
  if (warp == 0) {
    tmem_alloc(&tmem_base_sh, G::TMEM_COLS);
    tmem_relinquish();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tbase = tmem_base_sh;
  // one spectrum scratch (T blocked grids) per CTA of the launch, for MODE_OCC with omega
  float2* spec = args.spec ? args.spec + (size_t)blockIdx.x * Geo<n>::T * OrbBlk<n>::NBK : nullptr;
  pairconv_item<n, MODE, PPT, TSX, TC, BLK>(args, args.item0 + (int)blockIdx.x, smem4, tbase, true, spec);
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(tbase, G::TMEM_COLS);
}

// Dynamic shared memory requested per CTA: the grids, raised if needed so that no more CTAs
// become resident on an SM than its 512 TMEM columns can serve (tcgen05.alloc then never
// has to wait for another CTA).
template <int n>
constexpr size_t pairconv_smem_bytes() {
  constexpr size_t sm_smem = 233472;  // 228 KB of shared memory per SM
  constexpr int max_res = 512 / Geo<n>::TMEM_COLS;
  constexpr size_t floor_bytes = sm_smem / (size_t)(max_res + 1) + 2048;
  return Geo<n>::SMEM_BYTES > floor_bytes ? Geo<n>::SMEM_BYTES : floor_bytes;
}

// The same for the tensor-core variant: the grids, then the DFT tables.
template <int n, bool TC>
constexpr size_t pairconv_smem_request() {
  if constexpr (TC) {
    constexpr size_t need = Geo<n>::SMEM_BYTES + sizeof(TcTables<n>);
    static_assert(Geo<n>::SMEM_BYTES % 16 == 0, "the tables need 16-byte alignment");
    return need > pairconv_smem_bytes<n>() ? need : pairconv_smem_bytes<n>();
  } else {
    return pairconv_smem_bytes<n>();
  }
}

}  // namespace hse
