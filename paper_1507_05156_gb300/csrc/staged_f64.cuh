// staged_f64.cuh - plain FP64 (complex128) form of the Fock-like term, one kernel per step
// of Sec. II C, Eq. "Fock", on a batch of pair grids held in global memory:
//
//   pair_product  W[b] = conj(u_j) u_i            for b = (i, k', j) of one target k-point
//   fft_axis x3   forward 1-D DFTs along z, y, x  (register pencils, one thread each)
//   kernel_scale  W[b] *= v(|G+q|) * (-alpha f_j / N_k) / N
//   fft_axis x3   inverse 1-D DFTs along x, y, z
//   mul_acc       out[i] += sum_{k', j} u_j W[b]  (fixed order: deterministic)
//
// This is the FP64 reference form on the GPU and the denominator of the fused kernel's
// speedup.  It supports any grid whose axes are in the supported set.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_reg.cuh"

namespace hse {

struct StagedArgs {
  const double2* u_occ;  // [nk_occ][n_occ][N] occupied orbitals at the sampled k'
  const double2* u_tgt;  // [nk][n_tgt][N]  (or ybar)
  const double* occ;     // [nk_occ][n_occ]
  const double* vtab;    // [nq][N] FP64 kernel rows
  const int* qidx;       // [nk][nk_occ]
  double2* work;         // [nbatch][N]
  int nk_occ, n_occ, n_tgt, N;
  int k;                 // target k-point of this batch
  int kp0, nkp;          // k' range of this batch
  double scale;          // -alpha / (N_q N), N_q = nk_occ
};

// One thread per pencil of length L along an axis with element stride `inner`.
template <int L, int DIR>
__global__ void staged_fft_axis(double2* __restrict__ work, size_t nbatch, int N, int inner) {
  const int pencils = N / L;
  const size_t total = nbatch * pencils;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t bb = idx / pencils;
    const int p = (int)(idx - bb * pencils);
    const size_t base = bb * N + (size_t)(p / inner) * L * inner + (p % inner);
    cpx<double> v[L];
#pragma unroll
    for (int e = 0; e < L; ++e) {
      const double2 w = work[base + (size_t)e * inner];
      v[e] = {w.x, w.y};
    }
    fft<L, DIR, double>(v);
#pragma unroll
    for (int e = 0; e < L; ++e) work[base + (size_t)e * inner] = make_double2(v[e].x, v[e].y);
  }
}

// VJP w.r.t. the occupied orbitals (owner j at k-point kp, partners (k, i) for k in a chunk):
//   W1[b] = conj(u_j) u_i,  W2[b] = conj(u_j) ybar_i,  b = (j, kl, i), i fastest;
//   both transformed, scaled by v(|G+q|) (-alpha f_j / (N_q N)), q = k - kp, transformed back;
//   g_occ[kp][j] (+)= sum_{kl, i} conj(W1) ybar_i + u_i conj(W2).
struct StagedOccArgs {
  const double2* u_occ;  // [nk_occ][n_occ][N] occupied orbitals at the sampled k'
  const double2* u_tgt;  // [nk][n_tgt][N]
  const double2* ybar;   // [nk][n_tgt][N]
  const double* occ;     // [nk_occ][n_occ]
  const double* vtab;
  const int* qidx;       // [nk][nk_occ]
  double2* w1;           // [nbatch][N]
  double2* w2;           // [nbatch][N]
  int nk_occ, n_occ, n_tgt, N;
  int kp;                // owner k-point (index into the sampled k')
  int k0, nkc;           // partner (target) k range
  double scale;          // -alpha / (N_q N)
};

// Non-template stage kernels live in staged_f64.cu; these launch them on `stream`.
cudaError_t launch_staged_pair_product(const StagedArgs& a, cudaStream_t stream);
cudaError_t launch_staged_kernel_scale(const StagedArgs& a, cudaStream_t stream);
cudaError_t launch_staged_mul_acc(const StagedArgs& a, double2* out, int first, cudaStream_t stream);
cudaError_t launch_staged_occ_products(const StagedOccArgs& a, cudaStream_t stream);
cudaError_t launch_staged_occ_scale(const StagedOccArgs& a, cudaStream_t stream);
cudaError_t launch_staged_occ_acc(const StagedOccArgs& a, double2* g_occ, int first, cudaStream_t stream);

}  // namespace hse
