// ortho.cu - FP64 overlap matrices and Gram-Schmidt orthonormalisation of the orbitals.
//
// Orbitals u_{b,k} are cell-normalised: <a|b> = dV sum_r conj(u_a(r)) u_b(r), dV = Omega / N.
// The 4th-order Taylor propagator of Sec. II C is not unitary; the drift of the overlap matrix
// from the identity is the check of a propagation, and orthonormal sets are its input.  Both
// run in FP64 whatever the storage type (complex64 orbitals are widened on load and, for the
// orthonormalisation, rounded once when written back).
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.cuh"

namespace hse {
namespace {

constexpr int kOrthoThreads = 512;
constexpr int kOverlapThreads = 256;

__device__ __forceinline__ double2 widen(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 widen(double2 v) { return v; }
__device__ __forceinline__ void narrow(float2* p, double2 v) { *p = make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ void narrow(double2* p, double2 v) { *p = v; }

// Sum of v over the block (every thread gets it); red: 2 * (blockDim.x / 32) doubles.
__device__ __forceinline__ double2 block_sum2(double2 v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();  // red is free (a previous sum has been read by every thread)
  if (lane == 0) {
    red[2 * warp] = v.x;
    red[2 * warp + 1] = v.y;
  }
  __syncthreads();
  double2 s = make_double2(0.0, 0.0);
  for (int w = 0; w < nw; ++w) {
    s.x += red[2 * w];
    s.y += red[2 * w + 1];
  }
  return s;
}

// S[k][a][b] = dV sum_r conj(u_a) u_b and S[k][b][a] = conj of it (a real diagonal): block
// (pair a <= b, k).
template <typename C>
__global__ void __launch_bounds__(kOverlapThreads) overlap_kernel(const C* __restrict__ u, int nb, size_t N, double dV,
                                                                  double2* __restrict__ S) {
  __shared__ double red[2 * (kOverlapThreads / 32)];
  const int k = blockIdx.y;
  int pr = blockIdx.x, a = 0;
  while (pr >= nb - a) {  // pair index -> (a, b) with a <= b, row by row
    pr -= nb - a;
    ++a;
  }
  const int b = a + pr;
  const C* ua = u + ((size_t)k * nb + a) * N;
  const C* ub = u + ((size_t)k * nb + b) * N;
  double2 acc = make_double2(0.0, 0.0);
  for (size_t r = threadIdx.x; r < N; r += blockDim.x) {
    const double2 x = widen(ua[r]), y = widen(ub[r]);
    acc.x = fma(x.x, y.x, fma(x.y, y.y, acc.x));
    acc.y = fma(x.x, y.y, fma(-x.y, y.x, acc.y));
  }
  const double2 s = block_sum2(acc, red);
  if (threadIdx.x == 0) {
    if (a == b) {  // <a|a> is real: its imaginary part is rounding only
      S[((size_t)k * nb + a) * nb + a] = make_double2(dV * s.x, 0.0);
    } else {
      S[((size_t)k * nb + a) * nb + b] = make_double2(dV * s.x, dV * s.y);
      S[((size_t)k * nb + b) * nb + a] = make_double2(dV * s.x, -dV * s.y);
    }
  }
}

template <typename C>
__global__ void widen_orbitals(const C* __restrict__ u, double2* __restrict__ w, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    w[i] = widen(u[i]);
}

template <typename C>
__global__ void narrow_orbitals(const double2* __restrict__ w, C* __restrict__ u, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    narrow(u + i, w[i]);
}

// Modified Gram-Schmidt of the nb bands of k-point blockIdx.x in w (FP64, in place), `passes`
// times.  Band a: d = <w_b|w_a> for b = 0, 1, ... a-1 in turn, w_a -= d w_b, then
// w_a /= sqrt(<w_a|w_a>).  Each sweep over the grid applies one projection and accumulates the
// next inner product (with w_{b+1}, or the norm) from the updated values.  A band whose squared
// norm after the projections is at most rel2_min times its squared norm before them (or zero)
// is linearly dependent on the earlier ones: it is set to zero and the status word records
// HSE_ERR_SINGULAR.
__global__ void __launch_bounds__(kOrthoThreads) gram_schmidt_kernel(double2* __restrict__ w, int nb, size_t N,
                                                                      double dV, int passes, double rel2_min,
                                                                      int* status) {
  __shared__ double red[2 * (kOrthoThreads / 32)];
  double2* wk = w + (size_t)blockIdx.x * nb * N;
  for (int pass = 0; pass < passes; ++pass) {
    for (int a = 0; a < nb; ++a) {
      double2* wa = wk + (size_t)a * N;
      // the norm before the projections, and the first inner product
      double2 n0 = make_double2(0.0, 0.0), d0 = make_double2(0.0, 0.0);
      const double2* w0 = wk;
      for (size_t r = threadIdx.x; r < N; r += blockDim.x) {
        const double2 y = wa[r];
        n0.x = fma(y.x, y.x, fma(y.y, y.y, n0.x));
        if (a > 0) {
          const double2 x = w0[r];
          d0.x = fma(x.x, y.x, fma(x.y, y.y, d0.x));
          d0.y = fma(x.x, y.y, fma(-x.y, y.x, d0.y));
        }
      }
      const double norm0 = block_sum2(n0, red).x * dV;
      double2 d = block_sum2(d0, red);
      d.x *= dV;
      d.y *= dV;
      double norm = norm0;
      for (int b = 0; b < a; ++b) {
        const double2* wb = wk + (size_t)b * N;
        const bool last = b + 1 == a;
        const double2* wn = last ? wa : wk + (size_t)(b + 1) * N;
        double2 acc = make_double2(0.0, 0.0);
        for (size_t r = threadIdx.x; r < N; r += blockDim.x) {
          const double2 x = wb[r];
          double2 y = wa[r];
          y.x -= d.x * x.x - d.y * x.y;
          y.y -= d.x * x.y + d.y * x.x;
          wa[r] = y;
          if (last) {
            acc.x = fma(y.x, y.x, fma(y.y, y.y, acc.x));
          } else {
            const double2 z = wn[r];
            acc.x = fma(z.x, y.x, fma(z.y, y.y, acc.x));
            acc.y = fma(z.x, y.y, fma(-z.y, y.x, acc.y));
          }
        }
        const double2 s = block_sum2(acc, red);
        if (last) {
          norm = s.x * dV;
        } else {
          d = make_double2(s.x * dV, s.y * dV);
        }
      }
      const bool singular = !(norm > rel2_min * norm0) || !(norm0 > 0.0);
      const double scale = singular ? 0.0 : 1.0 / sqrt(norm);
      for (size_t r = threadIdx.x; r < N; r += blockDim.x) {
        const double2 y = wa[r];
        wa[r] = make_double2(y.x * scale, y.y * scale);
      }
      if (singular && threadIdx.x == 0 && status) atomicExch(status, kStatusSingular);
      __syncthreads();  // wa is final before later bands read it
    }
  }
}

unsigned grid_for_count(size_t count) {
  const size_t b = (count + 255) / 256;
  return (unsigned)(b < 152 * 16 ? (b ? b : 1) : 152 * 16);
}

}  // namespace

cudaError_t launch_overlap(bool c128, const void* u, int nk, int nb, size_t N, double dV, double2* S,
                           cudaStream_t stream) {
  const dim3 grid((unsigned)(nb * (nb + 1) / 2), (unsigned)nk);
  if (c128)
    overlap_kernel<double2><<<grid, kOverlapThreads, 0, stream>>>((const double2*)u, nb, N, dV, S);
  else
    overlap_kernel<float2><<<grid, kOverlapThreads, 0, stream>>>((const float2*)u, nb, N, dV, S);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_orthonormalize(bool c128, void* u, int nk, int nb, size_t N, double dV, double2* work, int* status,
                                  cudaStream_t stream) {
  const size_t count = (size_t)nk * nb * N;
  double2* w = c128 ? (double2*)u : work;
  if (!c128) {
    widen_orbitals<float2><<<grid_for_count(count), 256, 0, stream>>>((const float2*)u, w, count);
    count_launch();
  }
  // dependence threshold on the norm ratio: 1e-12 for FP64 data; 1e-5 for complex64, whose
  // rounding leaves about 1e-7 of any band outside the span of the others
  const double rel = c128 ? 1e-12 : 1e-5;
  gram_schmidt_kernel<<<(unsigned)nk, kOrthoThreads, 0, stream>>>(w, nb, N, dV, 2, rel * rel, status);
  count_launch();
  if (!c128) {
    narrow_orbitals<float2><<<grid_for_count(count), 256, 0, stream>>>(w, (float2*)u, count);
    count_launch();
  }
  return cudaGetLastError();
}

}  // namespace hse
