// kinetic.cu - the velocity-gauge kinetic term of the time-dependent Kohn-Sham Hamiltonian
// (Sec. II A, h_KS = (-i grad + A(t))^2 / 2 + ..., atomic units with e/c absorbed into A) on
// the periodic parts u_{b,k}:  (T u)(r) = sum_G 1/2 |G + k + A|^2 u~(G) e^{iG.r}.
// It is diagonal in G, so one forward 3-D FFT, a multiply and one inverse FFT per orbital.
//   complex64:  one fused kernel, the orbital's grid resident in shared memory (the pencil
//               stages of the pair-convolution kernel without the pair product);
//   complex128: the staged FP64 transforms on the output buffer.
#include "launch.cuh"

namespace hse {

namespace {

__host__ __device__ __forceinline__ int freq(int i, int n) { return i <= (n - 1) / 2 ? i : i - n; }

// 1/2 |G_m + k + A|^2 / N at grid index (i1, i2, i3); bf = reciprocal rows, kA = k + A
__device__ __forceinline__ float kin_factor(const float* bf, const float* kA, float inv_n, int n, int i1, int i2, int i3) {
  const float m1 = (float)freq(i1, n), m2 = (float)freq(i2, n), m3 = (float)freq(i3, n);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float g = m1 * bf[c] + m2 * bf[3 + c] + m3 * bf[6 + c] + kA[c];
    s = fmaf(g, g, s);
  }
  return 0.5f * s * inv_n;
}

template <int n>
__global__ void __launch_bounds__(Geo<n>::THREADS) kinetic_c64_kernel(const float2* __restrict__ u, float2* __restrict__ out,
                                                                    const KinArgs a) {
  using G = Geo<n>;
  extern __shared__ __align__(16) float4 smem4[];
  const int tid = threadIdx.x;
  const bool valid = tid < G::T * G::TS;
  const int slot = valid ? tid / G::TS : 0;
  const int t = valid ? tid - slot * G::TS : 0;
  float2* g = reinterpret_cast<float2*>(smem4) + slot * G::GRID_CPX;
  const int k = blockIdx.x / a.ntiles;
  const int band = (blockIdx.x - k * a.ntiles) * G::T + slot;
  const bool active = valid && band < a.nbands;
  const int bandc = active ? band : 0;
  const size_t obase = ((size_t)k * a.nbands + bandc) * G::N;
  float bf[9], kA[3];
#pragma unroll
  for (int c = 0; c < 9; ++c) bf[c] = (float)a.b[c];
#pragma unroll
  for (int c = 0; c < 3; ++c) kA[c] = (float)(a.kpts[3 * k + c] + a.A[c]);
  const float inv_n = 1.0f / (float)G::N;
#pragma unroll 1
  for (int ps = 0; ps < 2; ++ps) {
    const Pencil<n> pc(t + ps * G::TS);
    cpx<float> v[n];
    load_pencil_global<n>(v, u + obase + pc.zg);
    fft<n, -1, float>(v);
    if (valid) store_s<n, G::ZVEC>(v, g, pc.zs, 1);
  }
  __syncthreads();
  stage_y<n, -1>(g, t, valid);
  __syncthreads();
#pragma unroll 1
  for (int ps = 0; ps < 2; ++ps) {
    const int p = t + ps * G::TS;
    const Pencil<n> pc(p);
    cpx<float> v[n];
    load_s<n, 1>(v, g, pc.xs, G::Q);
    fft<n, -1, float>(v);
    const int i2 = p / n, i3 = p - i2 * n;  // X-stage pencil (y, z)
#pragma unroll
    for (int e = 0; e < n; ++e) {
      const float w = kin_factor(bf, kA, inv_n, n, e, i2, i3);
      v[e].x *= w;
      v[e].y *= w;
    }
    fft<n, +1, float>(v);
    if (valid) store_s<n, 1>(v, g, pc.xs, G::Q);
  }
  __syncthreads();
  stage_y<n, +1>(g, t, valid);
  __syncthreads();
#pragma unroll 1
  for (int ps = 0; ps < 2; ++ps) {
    const Pencil<n> pc(t + ps * G::TS);
    cpx<float> v[n];
    load_s<n, G::ZVEC>(v, g, pc.zs, 1);
    fft<n, +1, float>(v);
    if (active) {
      float4* o = reinterpret_cast<float4*>(out + obase + pc.zg);
#pragma unroll
      for (int e = 0; e < n / 2; ++e) o[e] = make_float4(v[2 * e].x, v[2 * e].y, v[2 * e + 1].x, v[2 * e + 1].y);
    }
  }
}

template <int n>
cudaError_t launch_kinetic_n(const float2* u, float2* out, const KinArgs& a, cudaStream_t stream) {
  constexpr size_t smem = Geo<n>::SMEM_BYTES;
  static bool attr_done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr_done[dev]) {
    cudaError_t err = cudaFuncSetAttribute(kinetic_c64_kernel<n>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    attr_done[dev] = true;
  }
  kinetic_c64_kernel<n><<<(unsigned)((size_t)a.nk * a.ntiles), Geo<n>::THREADS, smem, stream>>>(u, out, a);
  count_launch();
  return cudaGetLastError();
}

// FP64: out *= 1/2 |G + k + A|^2 / N per point (out already transformed forward)
__global__ void kinetic_scale_f64(double2* __restrict__ out, const KinArgs a) {
  const size_t N = (size_t)a.n1 * a.n2 * a.n3;
  const size_t total = (size_t)a.nk * a.nbands * N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % N);
    const int k = (int)(idx / ((size_t)a.nbands * N));
    const int i3 = r % a.n3, i2 = (r / a.n3) % a.n2, i1 = r / (a.n3 * a.n2);
    const double m1 = freq(i1, a.n1), m2 = freq(i2, a.n2), m3 = freq(i3, a.n3);
    double s = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double gc = m1 * a.b[c] + m2 * a.b[3 + c] + m3 * a.b[6 + c] + a.kpts[3 * k + c] + a.A[c];
      s += gc * gc;
    }
    const double w = 0.5 * s / (double)N;
    double2 v = out[idx];
    out[idx] = make_double2(v.x * w, v.y * w);
  }
}

}  // namespace

cudaError_t launch_kinetic_c64(int n, const float2* u, float2* out, const KinArgs& a, cudaStream_t stream) {
  switch (n) {
    case 4: return launch_kinetic_n<4>(u, out, a, stream);
    case 6: return launch_kinetic_n<6>(u, out, a, stream);
    case 8: return launch_kinetic_n<8>(u, out, a, stream);
    case 10: return launch_kinetic_n<10>(u, out, a, stream);
    case 12: return launch_kinetic_n<12>(u, out, a, stream);
    case 16: return launch_kinetic_n<16>(u, out, a, stream);
    case 18: return launch_kinetic_n<18>(u, out, a, stream);
    case 20: return launch_kinetic_n<20>(u, out, a, stream);
    case 24: return launch_kinetic_n<24>(u, out, a, stream);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_kinetic_f64(const double2* u, double2* out, const KinArgs& a, cudaStream_t stream) {
  const size_t N = (size_t)a.n1 * a.n2 * a.n3;
  const size_t nb = (size_t)a.nk * a.nbands;
  cudaError_t e = cudaMemcpyAsync(out, u, nb * N * sizeof(double2), cudaMemcpyDeviceToDevice, stream);
  const int dims[3] = {a.n1, a.n2, a.n3};
  const int inner[3] = {a.n2 * a.n3, a.n3, 1};
  for (int d = 2; d >= 0 && e == cudaSuccess; --d) e = launch_staged_fft(dims[d], -1, out, nb, (int)N, inner[d], stream);
  if (e == cudaSuccess) {
    const size_t total = nb * N;
    const unsigned blocks = (unsigned)((total + 255) / 256 < 152 * 64 ? (total + 255) / 256 : 152 * 64);
    kinetic_scale_f64<<<blocks, 256, 0, stream>>>(out, a);
    count_launch();
    e = cudaGetLastError();
  }
  for (int d = 0; d < 3 && e == cudaSuccess; ++d) e = launch_staged_fft(dims[d], +1, out, nb, (int)N, inner[d], stream);
  return e;
}

}  // namespace hse
