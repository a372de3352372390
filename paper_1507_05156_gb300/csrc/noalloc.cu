// noalloc.cu - hse_exchange_energy_noalloc: the exchange energy without any allocation.
//
// Some callers cannot call cudaMalloc: an application whose device memory is owned by
// another allocator (a framework's memory pool or a fixed per-process budget) that it may
// not grow, or a latency-critical loop in which cudaMalloc / cudaFree would synchronise the
// device.  hse_plan_create allocates (kernel tables, reduction scratch), so such callers
// cannot use the plan-based entry points.  This entry point needs no plan: its scratch is
// one file-scope __device__ array of fixed size, which every GPU that loads the library
// holds until the process exits.
//
// Scratch layout (bytes from the start of the array, each part 256-byte aligned):
//   status   int    [1]             device-side failure of this call (0: none)
//   qidx     int    [nk * nk]       row of (k, k'): k * nk + k'
//   vtab     float  [nk * nk][N]    v(|G + k - k'|) per ordered k-point pair
//   partial  double [nk * n_occ]    f_i Re<u_i, V_x u_i> per occupied orbital
// The k-points travel by value in the kernel parameters (at most kNoallocMaxK of them), so
// the call copies nothing from host memory.  The status word is cleared at the start of every
// call and every other part is fully overwritten before it is read, so nothing from a
// previous call leaks into the result.  Calls that overlap on the GPU (on different streams,
// or from different host threads) share this one array and race: serialise them.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "../../include/hse_fock.h"
#include "launch.cuh"

// The scratch array.  In host code this name is only a host-side stand-in; the device
// address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[HSE_NOALLOC_SCRATCH_BYTES];

namespace hse {

namespace {

constexpr int kMaxDevices = 64;
constexpr int kNoallocMaxK = 128;  // k-points passed by value (the scratch bounds nk below this anyway)
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_ptr[kMaxDevices] = {};
unsigned long long g_noalloc_ctx[kMaxDevices] = {};  // context the cached address belongs to

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Recip {
  double b[9];  // rows b1, b2, b3 (bohr^-1)
};

struct Kpts {
  double k[3 * kNoallocMaxK];  // Cartesian k-points (bohr^-1), [nk][3]
};

// Rows of v(|G+q|) for q = kpts[k] - kpts[k'], row k * nk + k', natural [x][y][z] order.
// Also clears the call's status word.
__global__ void noalloc_kernel_rows(const Kpts kp, int nk, int n, const Recip rb, double omega,
                                    int* __restrict__ qidx, float* __restrict__ vtab, int* __restrict__ status) {
  const size_t N = (size_t)n * n * n;
  const size_t rows = (size_t)nk * nk;
  const size_t total = rows * N;
  if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t row = idx / N;
    const int r = (int)(idx - row * N);
    const int k = (int)(row / nk);
    const int kq = (int)(row - (size_t)k * nk);
    if (r == 0) qidx[row] = (int)row;
    const int i3 = r % n, i2 = (r / n) % n, i1 = r / (n * n);
    const int m1 = (i1 <= (n - 1) / 2) ? i1 : i1 - n;
    const int m2 = (i2 <= (n - 1) / 2) ? i2 : i2 - n;
    const int m3 = (i3 <= (n - 1) / 2) ? i3 : i3 - n;
    double g2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double g = m1 * rb.b[c] + m2 * rb.b[3 + c] + m3 * rb.b[6 + c] + kp.k[3 * k + c] - kp.k[3 * kq + c];
      g2 += g * g;
    }
    const double w2 = omega * omega;
    const double x = g2 / (4.0 * w2);
    const double lim = kPi / w2;
    vtab[idx] = (float)((x == 0.0) ? lim : lim * (-expm1(-x) / x));
  }
}

// E_x = factor * sum of the partials, or NaN when a kernel of this call recorded a failed
// device-side wait or check in the status word (the partials are then incomplete).
__global__ void noalloc_reduce(const double* __restrict__ partial, int n, double factor, const int* __restrict__ status,
                               double* out) {
  __shared__ double sh[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = (*status != 0) ? __longlong_as_double(0x7ff8000000000000LL) : factor * sh[0];
}

// Identity of the calling thread's current context (0 if it cannot be read), so that an
// address cached for a device is looked up again after that device's context was replaced
// (cudaDeviceReset, a new primary context).
unsigned long long current_context_id() {
  static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess && fn)
      get_current = (PFN_cuCtxGetCurrent_v4000)fn;
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess && fn)
      get_id = (PFN_cuCtxGetId_v12000)fn;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

}  // namespace
}  // namespace hse

using namespace hse;

extern "C" int hse_exchange_energy_noalloc(const hse_problem* p, const void* u_occ, const double* occ, double* e_x,
                                           hse_stream_t stream) {
  if (!p || !u_occ || !occ || !e_x || !p->kpts) return HSE_ERR_INVALID_ARG;
  if (p->dtype != HSE_C64) return HSE_ERR_INVALID_ARG;
  const int n = p->grid[0];
  if (p->grid[1] != n || p->grid[2] != n || !pairconv_c64_supported(n)) return HSE_ERR_UNSUPPORTED_GRID;
  if (p->nk < 1 || p->n_occ < 1 || !(p->omega > 0.0) || !std::isfinite(p->omega) || !std::isfinite(p->alpha) ||
      !std::isfinite(p->spin_degeneracy))
    return HSE_ERR_INVALID_ARG;
  if ((((uintptr_t)u_occ) & 15u) != 0) return HSE_ERR_INVALID_ARG;
  if (p->nk_occ != 0) return HSE_ERR_INVALID_ARG;  // no down-sampling in the allocation-free form
  for (int i = 0; i < 3 * p->nk; ++i)
    if (!std::isfinite(p->kpts[i])) return HSE_ERR_INVALID_ARG;
  const double* A = p->lattice;
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (!(std::fabs(det) > 1e-12) || !std::isfinite(det)) return HSE_ERR_INVALID_ARG;

  // the problem must fit the fixed scratch array (and its k-points the kernel parameters)
  const size_t nk = (size_t)p->nk, N = (size_t)n * n * n;
  if (nk > (size_t)kNoallocMaxK) return HSE_ERR_INVALID_ARG;
  const size_t off_q = align256(sizeof(int));
  const size_t off_v = off_q + align256(nk * nk * sizeof(int));
  const size_t off_p = off_v + align256(nk * nk * N * sizeof(float));
  const size_t need = off_p + align256(nk * (size_t)p->n_occ * sizeof(double));
  if (need > (size_t)HSE_NOALLOC_SCRATCH_BYTES) return HSE_ERR_INVALID_ARG;

  // Set-up: the device address of the scratch array, looked up once per device (with that
  // device current) and again if the device's context has been replaced since.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HSE_ERR_CUDA;
  unsigned char* base = nullptr;
  {
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev] || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return HSE_ERR_CUDA;
      g_noalloc_ptr[dev] = (unsigned char*)ptr;
      g_noalloc_ctx[dev] = ctx;
    }
    base = g_noalloc_ptr[dev];
  }
  int* d_status = (int*)base;
  int* d_qidx = (int*)(base + off_q);
  float* d_vtab = (float*)(base + off_v);
  double* d_partial = (double*)(base + off_p);

  // reciprocal rows b_i = 2 pi (A^-1)^T, passed to the kernel by value
  double inv[9];
  inv[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  inv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  inv[3] = (A[5] * A[6] - A[3] * A[8]) / det;
  inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  inv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  inv[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  inv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  Recip rb;
  for (int i = 0; i < 3; ++i)
    for (int c = 0; c < 3; ++c) rb.b[3 * i + c] = 2.0 * kPi * inv[3 * c + i];
  Kpts kp;
  std::memset(&kp, 0, sizeof(kp));
  std::memcpy(kp.k, p->kpts, nk * 3 * sizeof(double));

  cudaStream_t st = (cudaStream_t)stream;
  const size_t total = nk * nk * N;
  const unsigned blocks = (unsigned)std::min<size_t>((total + 255) / 256, 152 * 32);
  noalloc_kernel_rows<<<blocks, 256, 0, st>>>(kp, p->nk, n, rb, p->omega, d_qidx, d_vtab, d_status);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return HSE_ERR_CUDA;

  PairArgs a{};
  a.own = (const float2*)u_occ;
  a.part = (const float2*)u_occ;
  a.partial = d_partial;
  a.occ = occ;
  a.occ_own = occ;
  a.vtab = d_vtab;
  a.qidx = d_qidx;
  a.nk_own = p->nk;
  a.nk_part = p->nk;
  a.n_own = p->n_occ;
  a.n_part = p->n_occ;
  a.n_occ = p->n_occ;
  a.scale = (float)(-p->alpha / ((double)p->nk * N));
  const int T = slots_for(n);
  a.ntiles = (p->n_occ + T - 1) / T;
  a.nsplit = 1;
  a.split_stride = 0;
  a.status = d_status;
  // the same test hook as the plans' (hse_status): the first partner copy is never issued
  const char* inj = std::getenv("HSE_INJECT_SKIP_FILL");
  a.inject = (inj && std::strcmp(inj, "1") == 0) ? 1 : 0;
  if (launch_pairconv_c64(n, MODE_ENERGY, a, 0, st) != cudaSuccess) return HSE_ERR_CUDA;

  const double dV = std::fabs(det) / (double)N;
  const double factor = 0.5 * p->spin_degeneracy * dV / p->nk;
  noalloc_reduce<<<1, 1024, 0, st>>>(d_partial, p->nk * p->n_occ, factor, d_status, e_x);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? HSE_OK : HSE_ERR_CUDA;
}
