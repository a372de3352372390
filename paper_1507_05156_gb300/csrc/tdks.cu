// tdks.cu - device pieces of the time propagation around the Fock operator (Sec. II A, II C):
//   * the Taylor-series accumulation of one fourth-order step,
//       term_n = (-i dt / n) (T term_{n-1} + V_x term_{n-1}),  out += term_n;
//   * the spatially averaged electric current (Eqs. current_dns / current_elec without the
//     nonlocal pseudopotential part):  J = -sum_{k,i} (g_s f_{i,k} / N_k) sum_G |c_G|^2 (G+k+A),
//     c_G = (1/N) sum_r u(r) e^{-iG.r}, reduced in FP64 per orbital and then in a fixed order;
//   * the Hartree potential of the orbitals' density (Sec. II A, Eq. tdks-h), FP64:
//       rho(r) = sum_{k,i} (g_s f_{i,k} / N_k) |u_{i,k}(r)|^2,
//       v_H = sum_{G != 0} 4 pi rho~(G) / |G|^2 e^{iG.r}  (G = 0 dropped: neutralising background).
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

// term = (-i s) (kin + vx + vloc prev),  out += term;  s = dt / n.  (-i s)(a + ib) = s b - i s a.
// prev: the previous term (may be the same array as term: each element is read, then
// written, by one thread); vloc: [N] real local potential or null.
template <typename C>
__global__ void taylor_accumulate(const C* __restrict__ kin, const C* __restrict__ vx, const C* prev,
                                  const double* __restrict__ vloc, size_t N, C* term, C* __restrict__ out,
                                  size_t count, double s_) {
  using T = typename Re<C>::T;
  const T s = (T)s_;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const C a = kin[i], b = vx[i];
    T hx = a.x + b.x, hy = a.y + b.y;
    if (vloc) {
      const T v = (T)vloc[i % N];
      const C p = prev[i];
      hx += v * p.x;
      hy += v * p.y;
    }
    C t;
    t.x = s * hy;
    t.y = -s * hx;
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

// rho[r] = (sum_o w_o |u_o[r]|^2, 0) with w_o = occ[o] * wscale, orbitals in a fixed order.
template <typename C>
__global__ void hartree_density(const C* __restrict__ u, const double* __restrict__ occ, size_t norb, size_t N,
                                double wscale, double2* __restrict__ rho) {
  for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < N; r += (size_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (size_t o = 0; o < norb; ++o) {
      const C v = u[o * N + r];
      const double x = (double)v.x, y = (double)v.y;
      acc += occ[o] * (x * x + y * y);
    }
    rho[r] = make_double2(wscale * acc, 0.0);
  }
}

// F(G) <- F(G) 4 pi / (N |G|^2), F(0) <- 0 (F: the unnormalised forward transform of rho)
__global__ void hartree_scale(double2* __restrict__ F, const CurArgs a) {
  const size_t N = (size_t)a.n1 * a.n2 * a.n3;
  for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < N; r += (size_t)gridDim.x * blockDim.x) {
    const int i3 = (int)(r % a.n3), i2 = (int)((r / a.n3) % a.n2), i1 = (int)(r / ((size_t)a.n3 * a.n2));
    const int m1 = i1 <= (a.n1 - 1) / 2 ? i1 : i1 - a.n1;
    const int m2 = i2 <= (a.n2 - 1) / 2 ? i2 : i2 - a.n2;
    const int m3 = i3 <= (a.n3 - 1) / 2 ? i3 : i3 - a.n3;
    double g2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double g = m1 * a.b[c] + m2 * a.b[3 + c] + m3 * a.b[6 + c];
      g2 += g * g;
    }
    const double f = g2 > 0.0 ? 4.0 * 3.14159265358979323846 / ((double)N * g2) : 0.0;
    const double2 v = F[r];
    F[r] = make_double2(v.x * f, v.y * f);
  }
}

__global__ void real_part(const double2* __restrict__ z, double* __restrict__ x, size_t N) {
  for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < N; r += (size_t)gridDim.x * blockDim.x)
    x[r] = z[r].x;
}

unsigned grid_for(size_t count) { return (unsigned)std::min<size_t>((count + 255) / 256, 152 * 16); }

}  // namespace

cudaError_t launch_taylor_accumulate(bool c128, const void* kin, const void* vx, const void* prev, const double* vloc,
                                     size_t N, void* term, void* out, size_t count, double s, cudaStream_t stream) {
  if (c128)
    taylor_accumulate<double2><<<grid_for(count), 256, 0, stream>>>((const double2*)kin, (const double2*)vx,
                                                                    (const double2*)prev, vloc, N, (double2*)term,
                                                                    (double2*)out, count, s);
  else
    taylor_accumulate<float2><<<grid_for(count), 256, 0, stream>>>((const float2*)kin, (const float2*)vx,
                                                                   (const float2*)prev, vloc, N, (float2*)term,
                                                                   (float2*)out, count, s);
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

cudaError_t launch_hartree(bool c128, const void* psi, const double* occ, const CurArgs& a, double spin_degeneracy,
                           double2* work, double* vh, cudaStream_t stream) {
  const size_t N = (size_t)a.n1 * a.n2 * a.n3;
  const size_t norb = (size_t)a.nk * a.nbands;
  const double wscale = spin_degeneracy / (double)a.nk;
  if (c128)
    hartree_density<double2><<<grid_for(N), 256, 0, stream>>>((const double2*)psi, occ, norb, N, wscale, work);
  else
    hartree_density<float2><<<grid_for(N), 256, 0, stream>>>((const float2*)psi, occ, norb, N, wscale, work);
  count_launch();
  cudaError_t e = cudaGetLastError();
  const int inner[3] = {a.n2 * a.n3, a.n3, 1};
  const int len[3] = {a.n1, a.n2, a.n3};
  for (int d = 2; d >= 0 && e == cudaSuccess; --d) e = launch_staged_fft(len[d], -1, work, 1, (int)N, inner[d], stream);
  if (e != cudaSuccess) return e;
  hartree_scale<<<grid_for(N), 256, 0, stream>>>(work, a);
  count_launch();
  e = cudaGetLastError();
  for (int d = 0; d < 3 && e == cudaSuccess; ++d) e = launch_staged_fft(len[d], +1, work, 1, (int)N, inner[d], stream);
  if (e != cudaSuccess) return e;
  real_part<<<grid_for(N), 256, 0, stream>>>(work, vh, N);
  count_launch();
  return cudaGetLastError();
}

}  // namespace hse
