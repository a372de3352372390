// Staged FP64 per-axis transform launches (one instantiation per supported axis length).
#include "launch.cuh"

namespace hse {

// batch element b = (i, kpl, j), j fastest
__global__ void staged_pair_product(const StagedArgs a) {
  const size_t total = (size_t)a.n_tgt * a.nkp * a.n_occ * a.N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % a.N);
    const size_t bidx = idx / a.N;
    const int j = (int)(bidx % a.n_occ);
    const int kpl = (int)((bidx / a.n_occ) % a.nkp);
    const int i = (int)(bidx / ((size_t)a.n_occ * a.nkp));
    const double2 ui = a.u_tgt[((size_t)a.k * a.n_tgt + i) * a.N + r];
    const double2 uj = a.u_occ[((size_t)(a.kp0 + kpl) * a.n_occ + j) * a.N + r];
    a.work[idx] = make_double2(uj.x * ui.x + uj.y * ui.y, uj.x * ui.y - uj.y * ui.x);
  }
}

__global__ void staged_kernel_scale(const StagedArgs a) {
  const size_t total = (size_t)a.n_tgt * a.nkp * a.n_occ * a.N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % a.N);
    const size_t bidx = idx / a.N;
    const int j = (int)(bidx % a.n_occ);
    const int kp = a.kp0 + (int)((bidx / a.n_occ) % a.nkp);
    const double s = a.vtab[(size_t)a.qidx[a.k * a.nk_occ + kp] * a.N + r] * a.scale * a.occ[kp * a.n_occ + j];
    double2 w = a.work[idx];
    w.x *= s;
    w.y *= s;
    a.work[idx] = w;
  }
}

// out[k][i][r] (+)= sum_{kpl, j} u_occ[kp][j][r] * W[(i, kpl, j)][r]
__global__ void staged_mul_acc(const StagedArgs a, double2* __restrict__ out, int first) {
  const size_t total = (size_t)a.n_tgt * a.N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % a.N);
    const int i = (int)(idx / a.N);
    double sx = 0.0, sy = 0.0;
    for (int kpl = 0; kpl < a.nkp; ++kpl) {
      for (int j = 0; j < a.n_occ; ++j) {
        const double2 uj = a.u_occ[((size_t)(a.kp0 + kpl) * a.n_occ + j) * a.N + r];
        const double2 w = a.work[(((size_t)i * a.nkp + kpl) * a.n_occ + j) * a.N + r];
        sx += uj.x * w.x - uj.y * w.y;
        sy += uj.x * w.y + uj.y * w.x;
      }
    }
    double2* o = out + ((size_t)a.k * a.n_tgt + i) * a.N + r;
    if (first) {
      *o = make_double2(sx, sy);
    } else {
      double2 c = *o;
      *o = make_double2(c.x + sx, c.y + sy);
    }
  }
}

// b = (j, kl, i), i fastest
__global__ void staged_occ_products(const StagedOccArgs a) {
  const size_t total = (size_t)a.n_occ * a.nkc * a.n_tgt * a.N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % a.N);
    const size_t b = idx / a.N;
    const int i = (int)(b % a.n_tgt);
    const int kl = (int)((b / a.n_tgt) % a.nkc);
    const int j = (int)(b / ((size_t)a.n_tgt * a.nkc));
    const int k = a.k0 + kl;
    const double2 uj = a.u_occ[((size_t)a.kp * a.n_occ + j) * a.N + r];
    const double2 ui = a.u_tgt[((size_t)k * a.n_tgt + i) * a.N + r];
    const double2 yi = a.ybar[((size_t)k * a.n_tgt + i) * a.N + r];
    a.w1[idx] = make_double2(uj.x * ui.x + uj.y * ui.y, uj.x * ui.y - uj.y * ui.x);
    a.w2[idx] = make_double2(uj.x * yi.x + uj.y * yi.y, uj.x * yi.y - uj.y * yi.x);
  }
}

__global__ void staged_occ_scale(const StagedOccArgs a) {
  const size_t total = (size_t)a.n_occ * a.nkc * a.n_tgt * a.N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % a.N);
    const size_t b = idx / a.N;
    const int kl = (int)((b / a.n_tgt) % a.nkc);
    const int j = (int)(b / ((size_t)a.n_tgt * a.nkc));
    const int k = a.k0 + kl;
    const double s = a.vtab[(size_t)a.qidx[k * a.nk_occ + a.kp] * a.N + r] * a.scale * a.occ[a.kp * a.n_occ + j];
    double2 w = a.w1[idx];
    a.w1[idx] = make_double2(w.x * s, w.y * s);
    w = a.w2[idx];
    a.w2[idx] = make_double2(w.x * s, w.y * s);
  }
}

// g_occ[kp][j][r] (+)= sum_{kl, i} conj(W1) ybar_i + u_i conj(W2)   (fixed order)
__global__ void staged_occ_acc(const StagedOccArgs a, double2* __restrict__ g_occ, int first) {
  const size_t total = (size_t)a.n_occ * a.N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % a.N);
    const int j = (int)(idx / a.N);
    double sx = 0.0, sy = 0.0;
    for (int kl = 0; kl < a.nkc; ++kl) {
      const int k = a.k0 + kl;
      for (int i = 0; i < a.n_tgt; ++i) {
        const size_t b = ((size_t)j * a.nkc + kl) * a.n_tgt + i;
        const double2 p = a.w1[b * a.N + r];
        const double2 q = a.w2[b * a.N + r];
        const double2 y = a.ybar[((size_t)k * a.n_tgt + i) * a.N + r];
        const double2 u = a.u_tgt[((size_t)k * a.n_tgt + i) * a.N + r];
        sx += p.x * y.x + p.y * y.y + u.x * q.x + u.y * q.y;
        sy += p.x * y.y - p.y * y.x + u.y * q.x - u.x * q.y;
      }
    }
    double2* o = g_occ + ((size_t)a.kp * a.n_occ + j) * a.N + r;
    if (first) {
      *o = make_double2(sx, sy);
    } else {
      const double2 c = *o;
      *o = make_double2(c.x + sx, c.y + sy);
    }
  }
}

namespace {
unsigned stage_blocks(size_t total) {
  size_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;  // grid-stride beyond this
  return (unsigned)(blocks ? blocks : 1);
}
}  // namespace

cudaError_t launch_staged_pair_product(const StagedArgs& a, cudaStream_t stream) {
  staged_pair_product<<<stage_blocks((size_t)a.n_tgt * a.nkp * a.n_occ * a.N), 256, 0, stream>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_staged_kernel_scale(const StagedArgs& a, cudaStream_t stream) {
  staged_kernel_scale<<<stage_blocks((size_t)a.n_tgt * a.nkp * a.n_occ * a.N), 256, 0, stream>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_staged_mul_acc(const StagedArgs& a, double2* out, int first, cudaStream_t stream) {
  staged_mul_acc<<<stage_blocks((size_t)a.n_tgt * a.N), 256, 0, stream>>>(a, out, first);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_staged_occ_products(const StagedOccArgs& a, cudaStream_t stream) {
  staged_occ_products<<<stage_blocks((size_t)a.n_occ * a.nkc * a.n_tgt * a.N), 256, 0, stream>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_staged_occ_scale(const StagedOccArgs& a, cudaStream_t stream) {
  staged_occ_scale<<<stage_blocks((size_t)a.n_occ * a.nkc * a.n_tgt * a.N), 256, 0, stream>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_staged_occ_acc(const StagedOccArgs& a, double2* g_occ, int first, cudaStream_t stream) {
  staged_occ_acc<<<stage_blocks((size_t)a.n_occ * a.N), 256, 0, stream>>>(a, g_occ, first);
  count_launch();
  return cudaGetLastError();
}

namespace {
template <int L>
cudaError_t run_axis(int dir, double2* work, size_t nbatch, int N, int inner, cudaStream_t stream) {
  const size_t total = nbatch * (size_t)(N / L);
  const int threads = 128;
  size_t blocks = (total + threads - 1) / threads;
  if (blocks > 152 * 64) blocks = 152 * 64;  // grid-stride beyond this
  if (blocks == 0) return cudaSuccess;
  if (dir < 0)
    staged_fft_axis<L, -1><<<(unsigned)blocks, threads, 0, stream>>>(work, nbatch, N, inner);
  else
    staged_fft_axis<L, +1><<<(unsigned)blocks, threads, 0, stream>>>(work, nbatch, N, inner);
  count_launch();
  return cudaGetLastError();
}
}  // namespace

#define HSE_AXIS_LIST(X) X(2) X(3) X(4) X(5) X(6) X(8) X(9) X(10) X(12) X(15) X(16) X(18) X(20) X(24) X(25) X(27) X(30) X(32)

bool staged_fft_supported(int L) {
  switch (L) {
#define HSE_CASE(L) case L:
    HSE_AXIS_LIST(HSE_CASE)
#undef HSE_CASE
    return true;
    default:
      return false;
  }
}

cudaError_t launch_staged_fft(int L, int dir, double2* work, size_t nbatch, int N, int inner, cudaStream_t stream) {
  switch (L) {
#define HSE_CASE(L) \
  case L:           \
    return run_axis<L>(dir, work, nbatch, N, inner, stream);
    HSE_AXIS_LIST(HSE_CASE)
#undef HSE_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace hse
