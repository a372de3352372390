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
// so HBM (in practice L2) traffic per pair is one read of each orbital pencil and the
// kernel row; the owner's accumulator lives in shared memory for the whole loop and is
// written once.  Thread t of a slot owns pencil (t / n, t % n) of whichever axis the
// stage transforms.  Shared-memory layout, per slot, structure-of-arrays float:
//   grid  G[x*Q + y*P + z]  (P odd, Q = n mod 32: bank-conflict-light pencils)
//   acc   A[(x*n + y)*P + z]
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_reg.cuh"

namespace hse {

__host__ __device__ constexpr int pitch_z(int n) { return (n % 2 == 0) ? n + 1 : n; }
__host__ __device__ constexpr int pitch_x(int n) {
  return n * pitch_z(n) + (((n - n * pitch_z(n)) % 32) + 32) % 32;
}

template <int n>
struct Geo {
  static constexpr int P = pitch_z(n);
  static constexpr int Q = pitch_x(n);
  static constexpr int NN = n * n;
  static constexpr int N = n * n * n;
  static constexpr int G_FLOATS = Q * n;
  static constexpr int A_FLOATS = NN * P;
  static constexpr int SLOT_FLOATS = 2 * G_FLOATS + 2 * A_FLOATS;
};

// Owner orbitals per CTA (slots), chosen so a CTA has 400-648 threads and fits smem.
__host__ __device__ constexpr int slots_for(int n) {
  return n <= 4 ? 32 : n <= 6 ? 16 : n <= 8 ? 8 : n <= 12 ? 4 : n <= 16 ? 2 : 1;
}

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
  const double* occ;    // [nk][n_occ] occupations
  const float* vtab;    // [nq][N] kernel rows v(|G+q|) (or d v / d omega)
  const int* qidx;      // [nk][nk] row of q = k - k' (first index k, second k')
  int nk, n_own, n_part, n_occ;
  int ntiles;           // ceil(n_own / slots)
  float scale;          // -alpha / (N_k * N): per-pair scale is scale * f
};

template <int n>
__device__ __forceinline__ void load_pencil_global(cpx<float> (&v)[n], const float2* __restrict__ p) {
  if constexpr (n % 2 == 0) {
    const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int e = 0; e < n / 2; ++e) {
      const float4 w = __ldg(p4 + e);
      v[2 * e] = {w.x, w.y};
      v[2 * e + 1] = {w.z, w.w};
    }
  } else {
#pragma unroll
    for (int e = 0; e < n; ++e) {
      const float2 w = __ldg(p + e);
      v[e] = {w.x, w.y};
    }
  }
}

template <int n>
__device__ __forceinline__ void load_s(cpx<float> (&v)[n], const float* re, const float* im, int base, int stride) {
#pragma unroll
  for (int e = 0; e < n; ++e) v[e] = {re[base + e * stride], im[base + e * stride]};
}

template <int n>
__device__ __forceinline__ void store_s(const cpx<float> (&v)[n], float* re, float* im, int base, int stride) {
#pragma unroll
  for (int e = 0; e < n; ++e) {
    re[base + e * stride] = v[e].x;
    im[base + e * stride] = v[e].y;
  }
}

// Stages Z(fwd) .. Z(inv) of one pair on the slot's smem grid.  On entry v holds the
// pair density of this thread's z-pencil; on exit it holds phi = K_q(rho) * s on the
// same z-pencil.  All threads of the CTA must call it together (it synchronises).
template <int n>
__device__ __forceinline__ void pair_chain(cpx<float> (&v)[n], float* gre, float* gim, int a, int b,
                                           const float* __restrict__ vrow, float s) {
  using G = Geo<n>;
  fft<n, -1, float>(v);
  store_s<n>(v, gre, gim, a * G::Q + b * G::P, 1);
  __syncthreads();
  // Y: thread owns (x = a, z = b)
  load_s<n>(v, gre, gim, a * G::Q + b, G::P);
  fft<n, -1, float>(v);
  store_s<n>(v, gre, gim, a * G::Q + b, G::P);
  __syncthreads();
  // X: thread owns (y = a, z = b); kernel row element (x, y, z) at x*n^2 + a*n + b
  load_s<n>(v, gre, gim, a * G::P + b, G::Q);
  fft<n, -1, float>(v);
#pragma unroll
  for (int e = 0; e < n; ++e) {
    const float w = __ldg(vrow + e * G::NN + a * n + b) * s;
    v[e].x *= w;
    v[e].y *= w;
  }
  fft<n, +1, float>(v);
  store_s<n>(v, gre, gim, a * G::P + b, G::Q);
  __syncthreads();
  // Y inverse
  load_s<n>(v, gre, gim, a * G::Q + b, G::P);
  fft<n, +1, float>(v);
  store_s<n>(v, gre, gim, a * G::Q + b, G::P);
  __syncthreads();
  // Z inverse
  load_s<n>(v, gre, gim, a * G::Q + b * G::P, 1);
  fft<n, +1, float>(v);
}

template <int n, int MODE>
__global__ void __launch_bounds__(slots_for(n) * n * n, 1) pairconv_c64_kernel(const PairArgs args) {
  using G = Geo<n>;
  constexpr int T = slots_for(n);
  extern __shared__ float smem[];
  const int slot = threadIdx.x / G::NN;
  const int t = threadIdx.x - slot * G::NN;
  const int a = t / n;
  const int b = t - a * n;
  float* gre = smem + slot * G::SLOT_FLOATS;
  float* gim = gre + G::G_FLOATS;
  float* are = gim + G::G_FLOATS;
  float* aim = are + G::A_FLOATS;

  const int k = blockIdx.x / args.ntiles;                         // owner k-point
  const int band = (blockIdx.x - k * args.ntiles) * T + slot;     // owner band
  const bool active = band < args.n_own;
  const int bandc = active ? band : 0;
  const size_t pencil = (size_t)t * n;                            // z-pencil offset in a grid
  const float2* own = args.own + ((size_t)k * args.n_own + bandc) * G::N + pencil;

  const int abase = t * G::P;
#pragma unroll
  for (int e = 0; e < n; ++e) {
    are[abase + e] = 0.f;
    aim[abase + e] = 0.f;
  }

  for (int kp = 0; kp < args.nk; ++kp) {
    // q = k_i - k_j: APPLY-like modes own i (at k), partners j at kp; OCC owns j (at k)
    const int qrow = (MODE == MODE_OCC) ? args.qidx[kp * args.nk + k] : args.qidx[k * args.nk + kp];
    const float* vrow = args.vtab + (size_t)qrow * G::N;
    for (int j = 0; j < args.n_part; ++j) {
      const size_t poff = ((size_t)kp * args.n_part + j) * G::N + pencil;
      if constexpr (MODE != MODE_OCC) {
        const float f = (float)args.occ[kp * args.n_occ + j];
        if (f == 0.f) continue;  // uniform over the CTA
        cpx<float> v[n], w[n];
        load_pencil_global<n>(v, own);
        load_pencil_global<n>(w, args.part + poff);
#pragma unroll
        for (int e = 0; e < n; ++e)  // conj(u_j) u_i
          v[e] = {w[e].x * v[e].x + w[e].y * v[e].y, w[e].x * v[e].y - w[e].y * v[e].x};
        pair_chain<n>(v, gre, gim, a, b, vrow, args.scale * f);
        load_pencil_global<n>(w, args.part + poff);
#pragma unroll
        for (int e = 0; e < n; ++e) {  // acc += u_j phi
          are[abase + e] += w[e].x * v[e].x - w[e].y * v[e].y;
          aim[abase + e] += w[e].x * v[e].y + w[e].y * v[e].x;
        }
      } else {
        const float f = (float)args.occ[k * args.n_occ + bandc];
        // chain 1: rho = conj(u_j) u_i -> phi; acc += conj(phi) ybar_i
        {
          cpx<float> v[n], w[n];
          load_pencil_global<n>(v, args.part + poff);
          load_pencil_global<n>(w, own);
#pragma unroll
          for (int e = 0; e < n; ++e)
            v[e] = {w[e].x * v[e].x + w[e].y * v[e].y, w[e].x * v[e].y - w[e].y * v[e].x};
          pair_chain<n>(v, gre, gim, a, b, vrow, args.scale * f);
          load_pencil_global<n>(w, args.part2 + poff);
#pragma unroll
          for (int e = 0; e < n; ++e) {
            are[abase + e] += v[e].x * w[e].x + v[e].y * w[e].y;
            aim[abase + e] += v[e].x * w[e].y - v[e].y * w[e].x;
          }
        }
        // chain 2: sigma = conj(u_j) ybar_i -> psibar; acc += u_i conj(psibar)
        {
          cpx<float> v[n], w[n];
          load_pencil_global<n>(v, args.part2 + poff);
          load_pencil_global<n>(w, own);
#pragma unroll
          for (int e = 0; e < n; ++e)
            v[e] = {w[e].x * v[e].x + w[e].y * v[e].y, w[e].x * v[e].y - w[e].y * v[e].x};
          pair_chain<n>(v, gre, gim, a, b, vrow, args.scale * f);
          load_pencil_global<n>(w, args.part + poff);
#pragma unroll
          for (int e = 0; e < n; ++e) {
            are[abase + e] += w[e].x * v[e].x + w[e].y * v[e].y;
            aim[abase + e] += w[e].y * v[e].x - w[e].x * v[e].y;
          }
        }
      }
    }
  }

  if constexpr (MODE == MODE_APPLY || MODE == MODE_OCC) {
    if (active) {
      float2* o = args.out + ((size_t)k * args.n_own + band) * G::N + pencil;
      if constexpr (n % 2 == 0) {
        float4* o4 = reinterpret_cast<float4*>(o);
#pragma unroll
        for (int e = 0; e < n / 2; ++e)
          o4[e] = make_float4(are[abase + 2 * e], aim[abase + 2 * e], are[abase + 2 * e + 1], aim[abase + 2 * e + 1]);
      } else {
#pragma unroll
        for (int e = 0; e < n; ++e) o[e] = make_float2(are[abase + e], aim[abase + e]);
      }
    }
  } else {
    // FP64 dot of the accumulator with u_i (ENERGY) or ybar_i (DOT), per owner.
    const float2* lhs = (MODE == MODE_ENERGY) ? own
                        : args.part2 + ((size_t)k * args.n_own + bandc) * G::N + pencil;
    cpx<float> w[n];
    load_pencil_global<n>(w, lhs);
    double d = 0.0;
#pragma unroll
    for (int e = 0; e < n; ++e) d += (double)w[e].x * (double)are[abase + e] + (double)w[e].y * (double)aim[abase + e];
    __syncthreads();  // the grid buffer is free now; reuse it for the per-thread partials
    double* red = reinterpret_cast<double*>(gre);
    red[t] = d;
    __syncthreads();
    if (t == 0 && active) {
      double sum = 0.0;
      for (int e = 0; e < G::NN; ++e) sum += red[e];
      if (MODE == MODE_ENERGY) sum *= args.occ[k * args.n_occ + band];
      args.partial[(size_t)k * args.n_own + band] = sum;
    }
  }
}

template <int n>
constexpr size_t pairconv_smem_bytes() {
  return (size_t)slots_for(n) * Geo<n>::SLOT_FLOATS * sizeof(float);
}

}  // namespace hse
