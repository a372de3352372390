// tdks.cu - device pieces of the time propagation around the Fock operator (Sec. II A, II C):
//   * the Taylor-series accumulation of one fourth-order step,
//       term_n = (-i dt / n) (T term_{n-1} + V_x term_{n-1}),  out += term_n;
//   * the spatially averaged electric current (Eqs. current_dns / current_elec without the
//     nonlocal pseudopotential part):  J = -sum_{k,i} (g_s f_{i,k} / N_k) sum_G |c_G|^2 (G+k+A),
//     c_G = (1/N) sum_r u(r) e^{-iG.r}, reduced in FP64 per orbital and then in a fixed order.
#include <algorithm>

#include "launch.cuh"

namespace hse {

namespace {

template <typename C>
struct Re;
template <>
struct Re<float2> { using T = float; };
template <>
struct Re<double2> { using T = double; };

// term = (-i s) (kin + vx),  out += term;  s = dt / n.  (-i s)(a + ib) = s b - i s a.
template <typename C>
__global__ void taylor_accumulate(const C* __restrict__ kin, const C* __restrict__ vx, C* __restrict__ term,
                                  C* __restrict__ out, size_t count, double s_) {
  using T = typename Re<C>::T;
  const T s = (T)s_;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const C a = kin[i], b = vx[i];
    C t;
    t.x = s * (a.y + b.y);
    t.y = -s * (a.x + b.x);
    term[i] = t;
    C o = out[i];
    o.x += t.x;
    o.y += t.y;
    out[i] = o;
  }
}

__global__ void widen_c64(const float2* __restrict__ u, double2* __restrict__ w, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const float2 a = u[i];
    w[i] = make_double2((double)a.x, (double)a.y);
  }
}

__device__ __forceinline__ int freq(int i, int n) { return i <= (n - 1) / 2 ? i : i - n; }

// partial[o][c] = sum_G |F(G)|^2 (G + k + A)_c for orbital o = (k, b) of the transformed
// batch F (unnormalised forward transform); one block per orbital.
__global__ void current_per_orbital(const double2* __restrict__ F, const CurArgs a, double* __restrict__ partial) {
  __shared__ double sh[3][256];
  const int o = blockIdx.x;
  const int k = o / a.nbands;
  const size_t N = (size_t)a.n1 * a.n2 * a.n3;
  double kA[3];
  for (int c = 0; c < 3; ++c) kA[c] = a.kpts[3 * k + c] + a.A[c];
  double s[3] = {0.0, 0.0, 0.0};
  for (size_t r = threadIdx.x; r < N; r += blockDim.x) {
    const int i3 = (int)(r % a.n3), i2 = (int)((r / a.n3) % a.n2), i1 = (int)(r / ((size_t)a.n3 * a.n2));
    const double m1 = freq(i1, a.n1), m2 = freq(i2, a.n2), m3 = freq(i3, a.n3);
    const double2 f = F[(size_t)o * N + r];
    const double w = f.x * f.x + f.y * f.y;
    for (int c = 0; c < 3; ++c) s[c] += w * (m1 * a.b[c] + m2 * a.b[3 + c] + m3 * a.b[6 + c] + kA[c]);
  }
  for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] = s[c];
  __syncthreads();
  for (int width = blockDim.x / 2; width > 0; width >>= 1) {
    if ((int)threadIdx.x < width)
      for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + width];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) partial[3 * (size_t)o + c] = sh[c][0];
}

// J_c = factor * sum_o f_o partial[o][c] (fixed order), factor = -g_s / (N_k N^2)
__global__ void current_combine(const double* __restrict__ partial, const double* __restrict__ occ, int norb,
                                double factor, double* __restrict__ J) {
  __shared__ double sh[3][256];
  double s[3] = {0.0, 0.0, 0.0};
  for (int o = threadIdx.x; o < norb; o += blockDim.x)
    for (int c = 0; c < 3; ++c) s[c] += occ[o] * partial[3 * (size_t)o + c];
  for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] = s[c];
  __syncthreads();
  for (int width = blockDim.x / 2; width > 0; width >>= 1) {
    if ((int)threadIdx.x < width)
      for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + width];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) J[c] = factor * sh[c][0];
}

unsigned grid_for(size_t count) { return (unsigned)std::min<size_t>((count + 255) / 256, 152 * 16); }

}  // namespace

cudaError_t launch_taylor_accumulate(bool c128, const void* kin, const void* vx, void* term, void* out, size_t count,
                                     double s, cudaStream_t stream) {
  if (c128)
    taylor_accumulate<double2><<<grid_for(count), 256, 0, stream>>>((const double2*)kin, (const double2*)vx,
                                                                    (double2*)term, (double2*)out, count, s);
  else
    taylor_accumulate<float2><<<grid_for(count), 256, 0, stream>>>((const float2*)kin, (const float2*)vx,
                                                                   (float2*)term, (float2*)out, count, s);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_current(bool c128, const void* psi, const double* occ, const CurArgs& a, double2* work,
                           double* partial, double spin_degeneracy, double* J, cudaStream_t stream) {
  const size_t N = (size_t)a.n1 * a.n2 * a.n3;
  const size_t norb = (size_t)a.nk * a.nbands;
  cudaError_t e;
  if (c128) {
    e = cudaMemcpyAsync(work, psi, norb * N * sizeof(double2), cudaMemcpyDeviceToDevice, stream);
  } else {
    widen_c64<<<grid_for(norb * N), 256, 0, stream>>>((const float2*)psi, work, norb * N);
    count_launch();
    e = cudaGetLastError();
  }
  const int inner[3] = {a.n2 * a.n3, a.n3, 1};
  const int len[3] = {a.n1, a.n2, a.n3};
  for (int d = 2; d >= 0 && e == cudaSuccess; --d) e = launch_staged_fft(len[d], -1, work, norb, (int)N, inner[d], stream);
  if (e != cudaSuccess) return e;
  current_per_orbital<<<(unsigned)norb, 256, 0, stream>>>(work, a, partial);
  count_launch();
  current_combine<<<1, 256, 0, stream>>>(partial, occ, (int)norb,
                                         -spin_degeneracy / ((double)a.nk * (double)N * (double)N), J);
  count_launch();
  return cudaGetLastError();
}

}  // namespace hse
