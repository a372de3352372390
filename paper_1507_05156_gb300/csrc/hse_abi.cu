// hse_abi.cu - the C ABI of include/hse_fock.h: plans, validation, dispatch, reductions.
//
// A plan holds, on the device:
//   * the q table: every distinct q = k - k' (k a target point, k' a point of the Fock sum:
//     all of them, or the sampled sub-mesh of a down-sampled plan; exact duplicates merged
//     after rounding to 1e-10 bohr^-1) and qidx[k][k'] -> row;
//   * for a down-sampled plan, the sampled rows of u_occ and occ gathered per call into
//     compact buffers (and the VJP w.r.t. them, scattered back to the full mesh);
//   * v(|G+q|) and d v/d omega per row, evaluated in FP64 (kept in FP64 for the staged
//     form, rounded once to FP32 for the fused form);
//   * reduction scratch: one double per owner orbital;
//   * for complex128 problems, the staged work batch and an FP64 result buffer;
//   * a status word that kernels set on a failed device-side check.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/hse_fock.h"
#include "launch.cuh"

namespace hse {
cudaError_t launch_pairconv_c64_small(int n, int mode, const PairArgs& args, int bps, cudaStream_t stream);
cudaError_t launch_pairconv_c64_mid(int n, int mode, const PairArgs& args, int bps, cudaStream_t stream);
cudaError_t launch_pairconv_c64_20(int mode, const PairArgs& args, int bps, cudaStream_t stream);
cudaError_t launch_pairconv_c64_24(int mode, const PairArgs& args, int bps, cudaStream_t stream);
int occupancy_pairconv_c64_small(int n, int mode, int bps);
int occupancy_pairconv_c64_mid(int n, int mode, int bps);
int occupancy_pairconv_c64_20(int mode, int bps);
int occupancy_pairconv_c64_24(int mode, int bps);
bool pencil_load_pairconv_c64_small(int n, int mode, int bps);
bool pencil_load_pairconv_c64_mid(int n, int mode, int bps);
bool pencil_load_pairconv_c64_20(int mode, int bps);
bool pencil_load_pairconv_c64_24(int mode, int bps);

bool pairconv_c64_pencil_load(int n, int mode, int bps) {
  if (n <= 12) return pencil_load_pairconv_c64_small(n, mode, bps);
  if (n <= 18) return pencil_load_pairconv_c64_mid(n, mode, bps);
  if (n == 20) return pencil_load_pairconv_c64_20(mode, bps);
  return pencil_load_pairconv_c64_24(mode, bps);
}

int pairconv_c64_occupancy(int n, int mode, int bps) {
  if (n <= 12) return occupancy_pairconv_c64_small(n, mode, bps);
  if (n <= 18) return occupancy_pairconv_c64_mid(n, mode, bps);
  if (n == 20) return occupancy_pairconv_c64_20(mode, bps);
  if (n == 24) return occupancy_pairconv_c64_24(mode, bps);
  return 0;
}

// For every cell with a k' split: final_out = sum of its split partials (ascending order,
// compensated).
__global__ void reduce_splits_batched(const BatchCell* __restrict__ cells, int ncells) {
  for (int c = 0; c < ncells; ++c) {
    const BatchCell& bc = cells[c];
    if (bc.pa.nsplit <= 1) continue;
    const size_t count4 = bc.pa.split_stride / 2;
    const float4* buf = reinterpret_cast<const float4*>(bc.pa.out);
    float4* out = reinterpret_cast<float4*>(bc.final_out);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count4; i += (size_t)gridDim.x * blockDim.x) {
      float4 a = buf[i], cs = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int sp = 1; sp < bc.pa.nsplit; ++sp) fold4(a, cs, buf[(size_t)sp * count4 + i], cs);
      out[i] = make_float4(a.x + cs.x, a.y + cs.y, a.z + cs.z, a.w + cs.w);
    }
  }
}

// Copy of norb orbitals in the pencil-blocked layout of the pencil-load kernel: the 16-byte
// chunk e (elements 2e, 2e + 1) of z-pencil p = 32 b + l goes to float4 (b n/2 + e) 32 + l of
// the orbital's nbk / 2 float4s; one thread per source chunk (coalesced reads).  The padding
// of a last partial block is left as it is (never read).
__global__ void to_pencil_blocks(float4* __restrict__ dst, const float4* __restrict__ src, int n, size_t nbk4,
                                 size_t norb) {
  const int h = n / 2;
  const size_t n4 = (size_t)n * n * h;  // float4 per orbital
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < norb * n4; i += (size_t)gridDim.x * blockDim.x) {
    const size_t o = i / n4;
    const size_t r = i - o * n4;
    const int p = (int)(r / h), e = (int)(r - (size_t)p * h);
    dst[o * nbk4 + ((size_t)(p >> 5) * h + e) * 32 + (p & 31)] = __ldg(src + i);
  }
}

// out[i] = sum_s buf[s * count + i], splits in ascending order (deterministic), compensated
// (TwoSum, as the k' groups inside a split)
__global__ void reduce_splits(float4* __restrict__ out, const float4* __restrict__ buf, int nsplit, size_t count4) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count4; i += (size_t)gridDim.x * blockDim.x) {
    float4 a = buf[i], c = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int sp = 1; sp < nsplit; ++sp) fold4(a, c, buf[(size_t)sp * count4 + i], c);
    out[i] = make_float4(a.x + c.x, a.y + c.y, a.z + c.z, a.w + c.w);
  }
}

static std::atomic<uint64_t> g_launches{0};
constexpr int kMaxBatchSplit = 4;

// The CUDA driver API's tensor-map encoder, obtained through the runtime (no link against libcuda).
cudaError_t make_partner_tmap(CUtensorMap* map, const void* base, int n, long long rows, int sp, int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return cudaErrorNotSupported;
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  if (rows <= 0 || rows > ((long long)1 << 32)) return cudaErrorInvalidValue;
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * n), (cuuint64_t)rows};  // floats of a pencil, pencils
  const cuuint64_t strides[1] = {(cuuint64_t)(2 * n) * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * sp), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

bool pairconv_c64_supported(int n) {
  switch (n) {
    case 4: case 6: case 8: case 10: case 12: case 16: case 18: case 20: case 24:
      return true;
    default:
      return false;
  }
}

cudaError_t launch_pairconv_c64(int n, int mode, const PairArgs& args, int bps, cudaStream_t stream) {
  if (n <= 12) return launch_pairconv_c64_small(n, mode, args, bps, stream);
  if (n <= 18) return launch_pairconv_c64_mid(n, mode, args, bps, stream);
  if (n == 20) return launch_pairconv_c64_20(mode, args, bps, stream);
  if (n == 24) return launch_pairconv_c64_24(mode, args, bps, stream);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// kernels owned by this TU
// ---------------------------------------------------------------------------

// v(|G+q|) = 4 pi / g^2 (1 - exp(-g^2 / 4 w^2)) = (pi / w^2) * (-expm1(-x) / x), x = g^2/4w^2,
// v(0) = pi / w^2; d v / d w = -(2 pi / w^3) exp(-x).  Rows in natural [x][y][z] order.
struct TableArgs {
  const double* qvec;  // [nq][3]
  int nq, n1, n2, n3;
  double b[9];         // reciprocal rows b1, b2, b3
  double omega;
  double* v64;
  double* dv64;
  float* v32;
  float* dv32;
};

__global__ void build_kernel_table(const TableArgs t) {
  const size_t N = (size_t)t.n1 * t.n2 * t.n3;
  const size_t total = N * t.nq;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int qi = (int)(idx / N);
    const int r = (int)(idx - (size_t)qi * N);
    const int i3 = r % t.n3;
    const int i2 = (r / t.n3) % t.n2;
    const int i1 = r / (t.n3 * t.n2);
    const int m1 = (i1 <= (t.n1 - 1) / 2) ? i1 : i1 - t.n1;
    const int m2 = (i2 <= (t.n2 - 1) / 2) ? i2 : i2 - t.n2;
    const int m3 = (i3 <= (t.n3 - 1) / 2) ? i3 : i3 - t.n3;
    double g[3];
    for (int c = 0; c < 3; ++c) g[c] = m1 * t.b[c] + m2 * t.b[3 + c] + m3 * t.b[6 + c] + t.qvec[3 * qi + c];
    const double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    const double w2 = t.omega * t.omega;
    const double x = g2 / (4.0 * w2);
    const double lim = kPi / w2;
    const double v = (x == 0.0) ? lim : lim * (-expm1(-x) / x);
    const double dv = -(2.0 * kPi / (w2 * t.omega)) * exp(-x);
    t.v64[idx] = v;
    t.dv64[idx] = dv;
    t.v32[idx] = (float)v;
    t.dv32[idx] = (float)dv;
  }
}

// out = factor * sum(partial[0..n)), fixed-order: deterministic.
__global__ void reduce_partials(const double* __restrict__ partial, int n, double factor, double* out) {
  __shared__ double sh[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = factor * sh[0];
}

// partial[o] = (weight ? w[o] : 1) * sum_r Re(conj(lhs[o][r]) rhs[o][r]), one block per owner o.
__global__ void dot_per_owner_f64(const double2* __restrict__ lhs, const double2* __restrict__ rhs, int N,
                                  const double* __restrict__ weight, double* __restrict__ partial) {
  __shared__ double sh[256];
  const size_t o = blockIdx.x;
  double s = 0.0;
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    const double2 a = lhs[o * N + r];
    const double2 b = rhs[o * N + r];
    s += a.x * b.x + a.y * b.y;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[o] = (weight ? weight[o] : 1.0) * sh[0];
}

// Sampled rows of the occupied set (down-sampling): dst[r] = src[idx[r]], rows of `words`
// 8-byte words.
__global__ void gather_rows(uint64_t* __restrict__ dst, const uint64_t* __restrict__ src, const int* __restrict__ idx,
                            int nrows, size_t words) {
  const size_t total = (size_t)nrows * words;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t r = i / words;
    dst[i] = src[(size_t)idx[r] * words + (i - r * words)];
  }
}

// Back to the full mesh: dst[r] = src[inv[r]] where inv[r] >= 0, else zeros.
__global__ void scatter_rows(uint64_t* __restrict__ dst, const uint64_t* __restrict__ src, const int* __restrict__ inv,
                             int nrows, size_t words) {
  const size_t total = (size_t)nrows * words;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t r = i / words;
    const int s = inv[r];
    dst[i] = s >= 0 ? src[(size_t)s * words + (i - r * words)] : 0ull;
  }
}

}  // namespace hse

using namespace hse;

// Roles of the fused kernel's owners, each with its own k' split: targets (apply, VJP
// w.r.t. u_tgt and omega), occupied orbitals at every target k-point (exchange energy),
// occupied orbitals at the sampled k' (VJP w.r.t. u_occ).
enum OwnerRole : int { ROLE_TGT = 0, ROLE_ENERGY = 1, ROLE_OCC = 2 };

// Streams (branches of the captured graph) of the per-cell batched form: each cell's
// single-cell launches go to the branch with the least work so far, so that a cell's last
// wave of CTAs shares the GPU with the next cells instead of leaving SMs idle.
constexpr int kCellBranches = 3;

struct hse_plan_s {
  hse_problem p;
  std::vector<double> kpts;
  int device = 0;
  int N = 0;
  int nq = 0;
  double dV = 0.0;
  double b[9] = {};
  int* qidx = nullptr;       // device [nk][nkq]
  double* qvec = nullptr;    // device [nq][3]
  double* dkpts = nullptr;   // device [nk][3]
  double* v64 = nullptr;     // device [nq][N]
  double* dv64 = nullptr;
  float* v32 = nullptr;
  float* dv32 = nullptr;
  double* partial = nullptr; // device [nk * max(n_occ, n_tgt)]
  int* status = nullptr;     // device status word
  // complex128 staged form
  double2* work = nullptr;   // [batch][N]
  size_t work_pairs = 0;
  double2* vx64 = nullptr;   // [nk][max(n_occ, n_tgt)][N]
  bool blocked = true;       // pencil-load launches read pencil-blocked copies (HSE_PENCIL_BLOCKS=0: no)
  int blocks_per_sm = 0;     // fused-kernel variant: 0 default, -1/-2 staged-partner layouts, 1/2/3/5 pencil loads,
                             // kTcVariant the tensor-core form (HSE_C64_TC)
  bool tc = false;           // created as HSE_C64_TC (p.dtype then reads HSE_C64)
  int inject = 0;            // test hook (HSE_INJECT_SKIP_FILL=1 at plan creation)
  long long alloc_count = 0;   // device allocations made by this plan so far (plan_malloc)
  long long fail_alloc_at = -1;  // test hook (HSE_FAIL_ALLOC_AT=k at plan creation): allocation k fails
  int nsplit[3] = {1, 1, 1};  // k'-loop splits of the fused kernel per OwnerRole
  float2* split_buf = nullptr;  // [nsplit][nk_own][n_own][N] partial outputs when nsplit > 1
  size_t split_buf_elems = 0;
  float2* comp_buf = nullptr;   // [nsplit][nk_own][n_own][2][blocked] running sums s, c (APPLY / OCC)
  // pencil-blocked copies of the orbital arrays a pencil-load launch reads (allocated on first
  // use, grown when a larger call comes)
  float2* blk_buf = nullptr;
  size_t blk_elems = 0;
  // MODE_OCC with the omega gradient fused in (allocated on first use): per CTA of a launch
  // chunk one spectrum of each owner slot, and one FP64 partial per work item
  float2* spec_buf = nullptr;
  size_t spec_elems = 0;
  double* wpartial = nullptr;
  size_t wpartial_elems = 0;
  // down-sampled Fock sum
  int nkq = 0;                  // k-points of the Fock sum: nk, or nk_occ when sampled
  bool sampled = false;
  std::vector<int> kocc;        // host [nkq] sampled k-point indices
  int* d_kocc = nullptr;        // device [nkq]
  int* d_kinv = nullptr;        // device [nk]: position in kocc, or -1
  void* u_sub = nullptr;        // device [nkq][n_occ][N] gathered occupied orbitals
  double* occ_sub = nullptr;    // device [nkq][n_occ]
  void* g_sub = nullptr;        // device [nkq][n_occ][N] VJP w.r.t. the sampled orbitals
  // time propagation (allocated on first use)
  void* tay[3] = {nullptr, nullptr, nullptr};  // Taylor step: term, T term, V_x term [nk][n_occ][N]
  double2* cur_work = nullptr;  // current: FP64 transforms [nk][n_occ][N]
  double* cur_partial = nullptr;  // current: [nk][n_occ][3]
  double2* hart_work = nullptr;   // Hartree potential: [N] FP64 transform
  double2* ortho_work = nullptr;  // orthonormalisation of complex64 orbitals: FP64 copy
  size_t ortho_elems = 0;
  // batched plans (hse_plan_create_batched)
  bool batched = false;
  std::vector<hse_plan> cells;          // one sub-plan (kernel tables) per cell
  std::vector<BatchCell> h_cells;       // launch arguments, pointers refreshed per call
  std::vector<float2*> cell_split;      // per cell [kMaxBatchSplit][nk][n_tgt][N]
  std::vector<float2*> cell_blk;        // pencil-load cells: blocked u_tgt then u_occ (else null)
  std::vector<float2*> cell_comp;       // per cell [min(kMaxBatchSplit, nk)][nk][n_tgt][2][blocked] running sums
  BatchCell* d_cells = nullptr;
  BatchItem* d_items = nullptr;         // staged-partner items, then pencil-load items
  int* d_counter = nullptr;             // [3]: one per list
  int nitems = 0;
  int nitems_staged = 0;
  int nitems_pencil = 0;
  int batch_split = 0;                  // autotuned k' split (0: not tuned yet)
  int batch_layout24 = kPencilOne;      // autotuned pencil layout of the 24^3 items
  bool batch_serial = false;            // autotuned: the two persistent kernels one after the other
  cudaStream_t side_stream = nullptr;   // the staged kernel's stream when both run at once
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool batch_percell = false;           // autotuned: every cell's single-cell launches, on parallel streams
  cudaStream_t cell_side[kCellBranches - 1] = {};  // per-cell form: the branches beside the main stream
  cudaEvent_t cell_join[kCellBranches - 1] = {};
  std::vector<const void*> call_ptrs;   // this call's u_occ, occ, u_tgt, vx_out of each cell
  std::vector<const void*> graph_ptrs;  // per-cell form: the call_ptrs the graph was captured with
  bool percell_warm = false;            // per-cell form: the sub-plans' scratch exists (one uncaptured run)
  int sms = 0;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t capture_stream = nullptr;
};

namespace {

constexpr long long kSpecCtas = 152 * 8;  // CTAs per launch chunk of the fused u_occ / omega pass

// NVTX range over one entry point (visible in Nsight Systems timelines; free without a tool).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// HSE_LOG=1: plan and autotune decisions on stderr
bool log_on() {
  const char* env = std::getenv("HSE_LOG");
  return env && std::atoi(env) != 0;
}

// Autotune cache (HSE_AUTOTUNE_CACHE=<file>): one line "<key>\t<k' split>" per batched
// problem, the key naming the GPU and every cell (grid side, k-points, bands).  Missing or
// unreadable files simply mean "not cached"; a failed write is ignored.
const char* autotune_path() {
  const char* p = std::getenv("HSE_AUTOTUNE_CACHE");
  return (p && *p) ? p : nullptr;
}

std::string autotune_key(hse_plan plan) {
  cudaDeviceProp prop{};
  std::string k = cudaGetDeviceProperties(&prop, plan->device) == cudaSuccess ? prop.name : "gpu";
  for (hse_plan c : plan->cells) {
    char buf[96];
    std::snprintf(buf, sizeof buf, "|%dx%dx%d,nk%d,o%d,t%d", c->p.grid[0], c->p.grid[1], c->p.grid[2], c->p.nk,
                  c->p.n_occ, c->p.n_tgt);
    k += buf;
  }
  return k;
}

int autotune_lookup(const std::string& key) {
  const char* path = autotune_path();
  if (!path) return 0;
  FILE* f = std::fopen(path, "r");
  if (!f) return 0;
  int found = 0;
  std::vector<char> line(1 << 16);
  while (std::fgets(line.data(), (int)line.size(), f)) {
    const char* tab = std::strchr(line.data(), '\t');
    if (!tab) continue;
    if ((size_t)(tab - line.data()) == key.size() && std::strncmp(line.data(), key.data(), key.size()) == 0) {
      const int v = std::atoi(tab + 1);
      const int split = v & 7;
      if (v > 0 && v < (1 << 11) && (split == 1 || split == 2 || split == 4)) found = v;  // the last entry wins
    }
  }
  std::fclose(f);
  return found;
}

void autotune_store(const std::string& key, int shape) {
  const char* path = autotune_path();
  if (!path || key.size() + 16 > (1 << 16)) return;
  if (FILE* f = std::fopen(path, "a")) {
    std::fprintf(f, "%s\t%d\n", key.c_str(), shape);
    std::fclose(f);
  }
}

// One point of the batched autotuner's search space, stored in the autotune cache as an int:
// bits 0-2 the k' split (1, 2 or 4), bit 3 the ragged 24^3 layout, bit 4 the kernels one after
// the other, bits 5-9 LayoutSeq for the staged sides 8, 16, 18, 20, 12 (12^3 then runs in the
// 512-thread staged kernel instead of its own LayoutOne kernel), bit 10 the per-cell form (every
// cell's single-cell launches on the branches of the graph; the other bits then unused).  Zero
// bits are the defaults, so a bare split (an older cache line) reads as the default shape.
constexpr int kShapeSides = 5;
struct BatchShape {
  int split = 1;
  int layout24 = kPencilOne;
  bool serial = false;
  int seq[kShapeSides] = {0, 0, 0, 0, 0};  // sides 8, 16, 18, 20, 12
  bool percell = false;
  int encode() const {
    int v = split | (layout24 == kPencilRagged ? 8 : 0) | (serial ? 16 : 0) | (percell ? 1024 : 0);
    for (int i = 0; i < kShapeSides; ++i) v |= seq[i] ? (32 << i) : 0;
    return v;
  }
  static BatchShape decode(int v) {
    BatchShape s;
    s.percell = (v & 1024) != 0;
    s.split = v & 7;
    s.layout24 = (v & 8) ? kPencilRagged : kPencilOne;
    s.serial = (v & 16) != 0;
    for (int i = 0; i < kShapeSides; ++i) s.seq[i] = (v >> (5 + i)) & 1;
    return s;
  }
};

int side_slot(int n) { return n == 8 ? 0 : n == 16 ? 1 : n == 18 ? 2 : n == 20 ? 3 : n == 12 ? 4 : -1; }

int cuda_fail(cudaError_t e) { return e == cudaSuccess ? HSE_OK : (e == cudaErrorMemoryAllocation ? HSE_ERR_NOMEM : HSE_ERR_CUDA); }

// Every device allocation of a plan goes through here.  Test hook: a plan created while the
// environment variable HSE_FAIL_ALLOC_AT=k is set has its k-th allocation (0-based, counted
// over the plan's life, creation included) fail as if the device were out of memory, without
// allocating anything, so that the clean-up of every failure path can be checked.
template <class T>
cudaError_t plan_malloc(hse_plan plan, T** p, size_t bytes) {
  if (plan->alloc_count++ == plan->fail_alloc_at) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc((void**)p, bytes);
}

// HSE_FAIL_ALLOC_AT, read when a plan is created (-1: the hook is off).
long long fail_alloc_from_env() {
  const char* env = std::getenv("HSE_FAIL_ALLOC_AT");
  return env ? std::atoll(env) : -1;
}

bool invert3(const double* A, double* inv) {
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (!(std::fabs(det) > 1e-12) || !std::isfinite(det)) return false;
  inv[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  inv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  inv[3] = (A[5] * A[6] - A[3] * A[8]) / det;
  inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  inv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  inv[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  inv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  return true;
}

size_t elem_bytes(int dtype) { return dtype == HSE_C128 ? 16 : 8; }

int validate_problem(const hse_problem* p) {
  if (!p) return HSE_ERR_INVALID_ARG;
  if (p->dtype != HSE_C64 && p->dtype != HSE_C128 && p->dtype != HSE_C64_TC) return HSE_ERR_INVALID_ARG;
  if (p->nk < 1 || p->n_occ < 1 || p->n_tgt < 1 || !p->kpts) return HSE_ERR_INVALID_ARG;
  if (!(p->omega > 0.0) || !std::isfinite(p->omega) || !std::isfinite(p->alpha) || !std::isfinite(p->spin_degeneracy))
    return HSE_ERR_INVALID_ARG;
  for (int d = 0; d < 3; ++d) {
    if (p->grid[d] < 2) return HSE_ERR_INVALID_ARG;
    if (!hse_grid_supported(p->grid[d], p->dtype)) return HSE_ERR_UNSUPPORTED_GRID;
  }
  if (p->dtype != HSE_C128 && (p->grid[0] != p->grid[1] || p->grid[1] != p->grid[2])) return HSE_ERR_UNSUPPORTED_GRID;
  for (int i = 0; i < 3 * p->nk; ++i)
    if (!std::isfinite(p->kpts[i])) return HSE_ERR_INVALID_ARG;
  if (p->nk_occ < 0 || p->nk_occ > p->nk || (p->nk_occ > 0 && !p->kocc)) return HSE_ERR_INVALID_ARG;
  if (p->nk_occ > 0) {
    std::vector<char> seen(p->nk, 0);
    for (int i = 0; i < p->nk_occ; ++i) {
      const int k = p->kocc[i];
      if (k < 0 || k >= p->nk || seen[k]) return HSE_ERR_INVALID_ARG;
      seen[k] = 1;
    }
  }
  // sizes must stay within int indexing of a single grid and the launch grid
  const double N = (double)p->grid[0] * p->grid[1] * p->grid[2];
  if (N > 1e8 || (double)p->nk * p->nk > 2e9 || (double)p->nk * std::max(p->n_occ, p->n_tgt) > 2e9)
    return HSE_ERR_INVALID_ARG;
  return HSE_OK;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  if (!a || !b || na == 0 || nb == 0) return false;
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

cudaStream_t S(hse_stream_t s) { return (cudaStream_t)s; }

}  // namespace

extern "C" {

int hse_grid_supported(int n, int dtype) {
  if (dtype == HSE_C64) return pairconv_c64_supported(n) ? 1 : 0;
  if (dtype == HSE_C128) return staged_fft_supported(n) ? 1 : 0;
  if (dtype == HSE_C64_TC) return n == 24 ? 1 : 0;
  return 0;
}

uint64_t hse_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char* hse_strerror(int code) {
  switch (code) {
    case HSE_OK: return "success";
    case HSE_ERR_INVALID_ARG: return "invalid argument";
    case HSE_ERR_UNSUPPORTED_GRID: return "unsupported grid (axis length or shape)";
    case HSE_ERR_ALIAS: return "output buffer overlaps an input";
    case HSE_ERR_CUDA: return "CUDA runtime error";
    case HSE_ERR_TIMEOUT: return "device-side wait timed out";
    case HSE_ERR_NOMEM: return "out of device memory";
    case HSE_ERR_DEVICE: return "device-side check failed";
    case HSE_ERR_SINGULAR: return "linearly dependent band in orthonormalisation";
    default: return "unknown error";
  }
}

int hse_plan_destroy(hse_plan plan) {
  if (!plan) return HSE_ERR_INVALID_ARG;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(plan->device);
  for (hse_plan c : plan->cells) hse_plan_destroy(c);
  for (float2* b : plan->cell_split) cudaFree(b);
  for (float2* b : plan->cell_blk) cudaFree(b);
  for (float2* b : plan->cell_comp) cudaFree(b);
  cudaFree(plan->d_cells);
  cudaFree(plan->d_items);
  cudaFree(plan->d_counter);
  if (plan->graph) cudaGraphExecDestroy(plan->graph);
  if (plan->capture_stream) cudaStreamDestroy(plan->capture_stream);
  if (plan->side_stream) cudaStreamDestroy(plan->side_stream);
  if (plan->ev_fork) cudaEventDestroy(plan->ev_fork);
  if (plan->ev_join) cudaEventDestroy(plan->ev_join);
  for (int b = 0; b < kCellBranches - 1; ++b) {
    if (plan->cell_side[b]) cudaStreamDestroy(plan->cell_side[b]);
    if (plan->cell_join[b]) cudaEventDestroy(plan->cell_join[b]);
  }
  cudaFree(plan->qidx);
  cudaFree(plan->qvec);
  cudaFree(plan->dkpts);
  cudaFree(plan->v64);
  cudaFree(plan->dv64);
  cudaFree(plan->v32);
  cudaFree(plan->dv32);
  cudaFree(plan->partial);
  cudaFree(plan->status);
  cudaFree(plan->work);
  cudaFree(plan->vx64);
  cudaFree(plan->split_buf);
  cudaFree(plan->comp_buf);
  cudaFree(plan->blk_buf);
  cudaFree(plan->spec_buf);
  cudaFree(plan->wpartial);
  cudaFree(plan->d_kocc);
  cudaFree(plan->d_kinv);
  cudaFree(plan->u_sub);
  cudaFree(plan->occ_sub);
  cudaFree(plan->g_sub);
  for (void* b : plan->tay) cudaFree(b);
  cudaFree(plan->cur_work);
  cudaFree(plan->cur_partial);
  cudaFree(plan->hart_work);
  cudaFree(plan->ortho_work);
  cudaSetDevice(prev);
  delete plan;
  return HSE_OK;
}

int hse_plan_create(hse_plan* out, const hse_problem* p) {
  const NvtxRange nvtx_range("hse_plan_create");
  if (!out) return HSE_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = validate_problem(p);
  if (rc) return rc;
  double ainv[9];
  if (!invert3(p->lattice, ainv)) return HSE_ERR_INVALID_ARG;

  hse_plan plan = new (std::nothrow) hse_plan_s();
  if (!plan) return HSE_ERR_NOMEM;
  plan->p = *p;
  if (p->dtype == HSE_C64_TC) {
    // complex64 throughout; the owner = target passes take the tensor-core kernel variant
    plan->p.dtype = HSE_C64;
    plan->tc = true;
  }
  plan->kpts.assign(p->kpts, p->kpts + 3 * p->nk);
  plan->p.kpts = plan->kpts.data();
  plan->sampled = p->nk_occ > 0;
  if (plan->sampled) {
    plan->kocc.assign(p->kocc, p->kocc + p->nk_occ);
  } else {
    plan->kocc.resize(p->nk);
    for (int k = 0; k < p->nk; ++k) plan->kocc[k] = k;
  }
  plan->nkq = (int)plan->kocc.size();
  plan->p.nk_occ = plan->sampled ? plan->nkq : 0;
  plan->p.kocc = plan->sampled ? plan->kocc.data() : nullptr;
  cudaGetDevice(&plan->device);
  if (const char* env = std::getenv("HSE_INJECT_SKIP_FILL")) plan->inject = std::atoi(env) == 1 ? 1 : 0;
  plan->fail_alloc_at = fail_alloc_from_env();
  if (const char* env = std::getenv("HSE_PENCIL_BLOCKS")) plan->blocked = std::atoi(env) != 0;
  if (const char* env = std::getenv("HSE_BLOCKS_PER_SM")) {
    const int v = std::atoi(env);
    plan->blocks_per_sm = (v < -2 || v > kOneVariant || v == kTcVariant) ? 0 : v;
  }
  if (plan->tc) plan->blocks_per_sm = kTcVariant;
  const int n1 = p->grid[0], n2 = p->grid[1], n3 = p->grid[2];
  plan->N = n1 * n2 * n3;
  // b_i = 2 pi (A^-1)^T rows: b_i[c] = 2 pi ainv[c][i]
  for (int i = 0; i < 3; ++i)
    for (int c = 0; c < 3; ++c) plan->b[3 * i + c] = 2.0 * kPi * ainv[3 * c + i];
  const double det = std::fabs(p->lattice[0] * (p->lattice[4] * p->lattice[8] - p->lattice[5] * p->lattice[7]) -
                               p->lattice[1] * (p->lattice[3] * p->lattice[8] - p->lattice[5] * p->lattice[6]) +
                               p->lattice[2] * (p->lattice[3] * p->lattice[7] - p->lattice[4] * p->lattice[6]));
  plan->dV = det / plan->N;

  // distinct q = k - k' over target points k and the points k' of the Fock sum
  const int nk = p->nk, nkq = plan->nkq;
  std::vector<int> qidx((size_t)nk * nkq);
  std::vector<double> qvec;
  std::map<std::array<long long, 3>, int> seen;
  for (int k = 0; k < nk; ++k) {
    for (int kp = 0; kp < nkq; ++kp) {
      double q[3];
      std::array<long long, 3> key;
      for (int c = 0; c < 3; ++c) {
        q[c] = plan->kpts[3 * k + c] - plan->kpts[3 * plan->kocc[kp] + c];
        key[c] = std::llround(q[c] * 1e10);
      }
      auto it = seen.find(key);
      if (it == seen.end()) {
        const int id = (int)(qvec.size() / 3);
        seen.emplace(key, id);
        qvec.insert(qvec.end(), q, q + 3);
        qidx[(size_t)k * nkq + kp] = id;
      } else {
        qidx[(size_t)k * nkq + kp] = it->second;
      }
    }
  }
  plan->nq = (int)(qvec.size() / 3);
  const size_t N = plan->N, nq = plan->nq;
  const int nown = std::max(p->n_occ, p->n_tgt);
  cudaError_t e = cudaSuccess;
#define HSE_TRY(call)              \
  do {                             \
    e = (call);                    \
    if (e != cudaSuccess) {        \
      rc = cuda_fail(e);           \
      hse_plan_destroy(plan);      \
      return rc;                   \
    }                              \
  } while (0)
  HSE_TRY(plan_malloc(plan, &plan->qidx, qidx.size() * sizeof(int)));
  HSE_TRY(plan_malloc(plan, &plan->qvec, qvec.size() * sizeof(double)));
  HSE_TRY(plan_malloc(plan, &plan->v64, nq * N * sizeof(double)));
  HSE_TRY(plan_malloc(plan, &plan->dv64, nq * N * sizeof(double)));
  HSE_TRY(plan_malloc(plan, &plan->v32, nq * N * sizeof(float)));
  HSE_TRY(plan_malloc(plan, &plan->dv32, nq * N * sizeof(float)));
  if (plan->p.dtype == HSE_C64) {
    // Split the k' loop so that the work items fill the resident CTA slots in nearly whole
    // waves; the partial outputs are summed by reduce_splits.
    int sms = 0;
    HSE_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, plan->device));
    const int occ_blocks = std::max(1, pairconv_c64_occupancy(n1, MODE_APPLY, plan->blocks_per_sm));
    const long long slots = (long long)sms * occ_blocks;
    // per OwnerRole: owner bands, owner k-points, partner k-points, partner bands
    const int owners[3] = {p->n_tgt, p->n_occ, p->n_occ};
    const int k_own[3] = {nk, nk, nkq};
    const int k_part[3] = {nkq, nkq, nk};
    const int b_part[3] = {p->n_occ, p->n_occ, p->n_tgt};
    size_t buf = 0, comp = 0;
    for (int o = 0; o < 3; ++o) {
      const int T = slots_for(n1);
      const long long items = (long long)k_own[o] * ((owners[o] + T - 1) / T);
      // the staged-partner kernel (roles with owner = target) caches an item's occupations:
      // at most kOccCache partners per item
      const int ns_cap = std::min(8, k_part[o]);
      const int ns_min =
          (plan->blocks_per_sm <= 0 && o != ROLE_OCC)
              ? std::min(ns_cap, std::max(1, (int)(((long long)k_part[o] * b_part[o] + kOccCache - 1) / kOccCache)))
              : 1;
      double best_eff = 0.0;
      int best = ns_min;
      for (int ns = ns_min; ns <= ns_cap; ++ns) {
        const long long it = items * ns;
        const long long waves = (it + slots - 1) / slots;
        const double eff = (double)it / (double)(waves * slots);
        if (eff > best_eff + 0.02) {
          best_eff = eff;
          best = ns;
        }
      }
      const size_t need = (best > 1 && o != ROLE_ENERGY) ? (size_t)best * k_own[o] * owners[o] * N : 0;
      if (need * sizeof(float2) > ((size_t)4 << 30)) best = 1;  // keep split buffers modest
      plan->nsplit[o] = best;
      if (best > 1) buf = std::max(buf, need);
      if (o != ROLE_ENERGY) comp = std::max(comp, (size_t)best * k_own[o] * owners[o] * 2 * blocked_stride(n1));
    }
    if (buf) {
      HSE_TRY(plan_malloc(plan, &plan->split_buf, buf * sizeof(float2)));
      plan->split_buf_elems = buf;
    }
    HSE_TRY(plan_malloc(plan, &plan->comp_buf, comp * sizeof(float2)));
  }
  {
    const size_t np = std::max((size_t)plan->nsplit[ROLE_TGT] * nk * p->n_tgt,
                               (size_t)plan->nsplit[ROLE_ENERGY] * nk * p->n_occ);
    HSE_TRY(plan_malloc(plan, &plan->partial, std::max(np, (size_t)nk * nown) * sizeof(double)));
  }
  if (plan->sampled) {
    std::vector<int> kinv(nk, -1);
    for (int i = 0; i < nkq; ++i) kinv[plan->kocc[i]] = i;
    const size_t sub_bytes = (size_t)nkq * p->n_occ * N * elem_bytes(p->dtype);
    HSE_TRY(plan_malloc(plan, &plan->d_kocc, (size_t)nkq * sizeof(int)));
    HSE_TRY(plan_malloc(plan, &plan->d_kinv, (size_t)nk * sizeof(int)));
    HSE_TRY(cudaMemcpy(plan->d_kocc, plan->kocc.data(), (size_t)nkq * sizeof(int), cudaMemcpyHostToDevice));
    HSE_TRY(cudaMemcpy(plan->d_kinv, kinv.data(), (size_t)nk * sizeof(int), cudaMemcpyHostToDevice));
    HSE_TRY(plan_malloc(plan, &plan->u_sub, sub_bytes));
    HSE_TRY(plan_malloc(plan, &plan->g_sub, sub_bytes));
    HSE_TRY(plan_malloc(plan, &plan->occ_sub, (size_t)nkq * p->n_occ * sizeof(double)));
  }
  HSE_TRY(plan_malloc(plan, &plan->status, sizeof(int)));
  HSE_TRY(cudaMemset(plan->status, 0, sizeof(int)));
  HSE_TRY(cudaMemcpy(plan->qidx, qidx.data(), qidx.size() * sizeof(int), cudaMemcpyHostToDevice));
  HSE_TRY(cudaMemcpy(plan->qvec, qvec.data(), qvec.size() * sizeof(double), cudaMemcpyHostToDevice));
  HSE_TRY(plan_malloc(plan, &plan->dkpts, (size_t)nk * 3 * sizeof(double)));
  HSE_TRY(cudaMemcpy(plan->dkpts, plan->kpts.data(), (size_t)nk * 3 * sizeof(double), cudaMemcpyHostToDevice));
  if (plan->p.dtype == HSE_C128) {
    // staged batch: all (i, k', j) of one k in chunks of k' up to ~512 MB
    // the energy path runs the staged form with the occupied set as targets
    const size_t per_kp = (size_t)nown * p->n_occ;
    size_t nkp = std::max<size_t>(1, ((size_t)512 << 20) / (per_kp * N * sizeof(double2)));
    nkp = std::min<size_t>(nkp, (size_t)nkq);
    // at least two occupied x target batches: the VJP w.r.t. u_occ runs two at a time
    plan->work_pairs = std::max(nkp * per_kp, 2 * (size_t)p->n_occ * p->n_tgt);
    HSE_TRY(plan_malloc(plan, &plan->work, plan->work_pairs * N * sizeof(double2)));
    HSE_TRY(plan_malloc(plan, &plan->vx64, (size_t)nk * nown * N * sizeof(double2)));
  }
  TableArgs t{};
  t.qvec = plan->qvec;
  t.nq = plan->nq;
  t.n1 = n1;
  t.n2 = n2;
  t.n3 = n3;
  std::memcpy(t.b, plan->b, sizeof(t.b));
  t.omega = p->omega;
  t.v64 = plan->v64;
  t.dv64 = plan->dv64;
  t.v32 = plan->v32;
  t.dv32 = plan->dv32;
  const size_t total = nq * N;
  const unsigned blocks = (unsigned)std::min<size_t>((total + 255) / 256, 152 * 32);
  build_kernel_table<<<blocks, 256>>>(t);
  count_launch();
  HSE_TRY(cudaGetLastError());
  HSE_TRY(cudaDeviceSynchronize());
#undef HSE_TRY
  if (log_on()) {
    const bool c64 = plan->p.dtype == HSE_C64;
    std::fprintf(stderr,
                 "hse: plan grid %dx%dx%d %s nk %d (Fock sum over %d) n_occ %d n_tgt %d: %d distinct q; "
                 "k' splits target %d energy %d occupied %d; apply kernel %s; pencil-blocked copies %s\n",
                 n1, n2, n3, c64 ? "complex64" : "complex128", nk, nkq, p->n_occ, p->n_tgt, plan->nq,
                 plan->nsplit[ROLE_TGT], plan->nsplit[ROLE_ENERGY], plan->nsplit[ROLE_OCC],
                 !c64 ? "staged FP64" : (pairconv_c64_pencil_load(n1, MODE_APPLY, plan->blocks_per_sm)
                                             ? (plan->tc ? "pencil-load, tensor-core Y/X" : "pencil-load")
                                                                                                    : "staged-partner"),
                 plan->blocked ? "on" : "off");
  }
  *out = plan;
  return HSE_OK;
}

int hse_status(hse_plan plan, hse_stream_t stream) {
  if (!plan) return HSE_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(S(stream));
  if (e != cudaSuccess) return HSE_ERR_CUDA;
  int st = 0;
  e = cudaMemcpy(&st, plan->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return HSE_ERR_CUDA;
  if (st != 0) {
    cudaMemset(plan->status, 0, sizeof(int));
    return (st == HSE_ERR_TIMEOUT || st == HSE_ERR_SINGULAR) ? st : HSE_ERR_DEVICE;
  }
  return HSE_OK;
}

}  // extern "C"

namespace {

// Owners are targets at every k-point; partners the occupied orbitals of the Fock sum.
PairArgs base_args(hse_plan plan) {
  PairArgs a{};
  a.occ = nullptr;
  a.occ_own = nullptr;
  a.vtab = plan->v32;
  a.qidx = plan->qidx;
  a.nk_own = plan->p.nk;
  a.nk_part = plan->nkq;
  a.n_occ = plan->p.n_occ;
  a.scale = (float)(-plan->p.alpha / ((double)plan->nkq * plan->N));
  a.status = plan->status;
  a.inject = plan->inject;
  return a;
}

int role_of(int mode) { return mode == MODE_ENERGY ? ROLE_ENERGY : (mode == MODE_OCC ? ROLE_OCC : ROLE_TGT); }

// Blocked layouts of the orbital arrays a pencil-load launch reads (own, part and, for
// MODE_DOT / MODE_OCC, part2), in the plan's scratch; an array given twice is copied once.
int to_blocked(hse_plan plan, int mode, PairArgs& a, cudaStream_t st) {
  const int n = plan->p.grid[0];
  const size_t nbk = blocked_stride(n);
  struct Arr {
    const float2** ptr;
    size_t norb;
  };
  Arr arrs[3] = {{&a.own, (size_t)a.nk_own * a.n_own}, {&a.part, (size_t)a.nk_part * a.n_part}, {&a.part2, 0}};
  if (mode == MODE_DOT) arrs[2].norb = (size_t)a.nk_own * a.n_own;
  if (mode == MODE_OCC) arrs[2].norb = (size_t)a.nk_part * a.n_part;
  size_t need = 0;
  for (const Arr& r : arrs) need += r.norb * nbk;
  if (need > plan->blk_elems) {
    cudaFree(plan->blk_buf);
    plan->blk_buf = nullptr;
    plan->blk_elems = 0;
    const cudaError_t e = plan_malloc(plan, &plan->blk_buf, need * sizeof(float2));
    if (e != cudaSuccess) return cuda_fail(e);
    plan->blk_elems = need;
  }
  const float2* src[3] = {a.own, a.part, a.part2};
  const float2* dst[3] = {nullptr, nullptr, nullptr};
  size_t off = 0;
  for (int i = 0; i < 3; ++i) {
    if (!arrs[i].norb) continue;
    for (int j = 0; j < i; ++j)
      if (arrs[j].norb == arrs[i].norb && src[j] == src[i]) dst[i] = dst[j];
    if (!dst[i]) {
      float2* d = plan->blk_buf + off;
      off += arrs[i].norb * nbk;
      const size_t count4 = arrs[i].norb * plan->N / 2;
      const unsigned blocks = (unsigned)std::min<size_t>((count4 + 255) / 256, 152 * 16);
      to_pencil_blocks<<<blocks, 256, 0, st>>>((float4*)d, (const float4*)src[i], n, nbk / 2, arrs[i].norb);
      count_launch();
      dst[i] = d;
    }
    *arrs[i].ptr = dst[i];
  }
  a.blk = 1;
  return cuda_fail(cudaGetLastError());
}

int run_pairconv(hse_plan plan, int mode, PairArgs a, int n_own, cudaStream_t st) {
  const int n = plan->p.grid[0];
  const int T = slots_for(n);
  a.n_own = n_own;
  if (pairconv_c64_pencil_load(n, mode, plan->blocks_per_sm) && plan->blocked) {
    const int rc = to_blocked(plan, mode, a, st);
    if (rc) return rc;
  }
  a.ntiles = (n_own + T - 1) / T;
  a.nsplit = plan->nsplit[role_of(mode)];
  const size_t count = (size_t)a.nk_own * n_own * plan->N;
  float2* final_out = a.out;
  a.comp = plan->comp_buf;
  if (mode == MODE_ENERGY || mode == MODE_DOT) {
    a.split_stride = (size_t)a.nk_own * n_own;  // doubles between the splits' partials
  } else {
    a.split_stride = count;
    if (a.nsplit > 1) a.out = plan->split_buf;
  }
  cudaError_t e = cudaSuccess;
  if (mode == MODE_OCC && a.vtab2) {
    // the omega gradient fused into the u_occ pass: launches of at most kSpecCtas CTAs, each
    // CTA with its own spectrum scratch, and one FP64 partial per item
    const long long items = (long long)a.nsplit * a.nk_own * a.ntiles;
    const size_t per_cta = (size_t)slots_for(n) * blocked_stride(n);
    const size_t spec_need = (size_t)std::min<long long>(items, kSpecCtas) * per_cta;
    if (spec_need > plan->spec_elems) {
      cudaFree(plan->spec_buf);
      plan->spec_buf = nullptr;
      plan->spec_elems = 0;
      e = plan_malloc(plan, &plan->spec_buf, spec_need * sizeof(float2));
      if (e != cudaSuccess) return cuda_fail(e);
      plan->spec_elems = spec_need;
    }
    if ((size_t)items > plan->wpartial_elems) {
      cudaFree(plan->wpartial);
      plan->wpartial = nullptr;
      plan->wpartial_elems = 0;
      e = plan_malloc(plan, &plan->wpartial, (size_t)items * sizeof(double));
      if (e != cudaSuccess) return cuda_fail(e);
      plan->wpartial_elems = (size_t)items;
    }
    a.spec = plan->spec_buf;
    a.partial2 = plan->wpartial;
    for (long long c0 = 0; c0 < items && e == cudaSuccess; c0 += kSpecCtas) {
      a.item0 = (int)c0;
      a.item_count = (int)std::min<long long>(kSpecCtas, items - c0);
      e = launch_pairconv_c64(n, mode, a, plan->blocks_per_sm, st);
    }
  } else {
    e = launch_pairconv_c64(n, mode, a, plan->blocks_per_sm, st);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  if ((mode == MODE_APPLY || mode == MODE_OCC) && a.nsplit > 1) {
    const size_t count4 = count / 2;  // N is even: whole float4 pairs
    const unsigned blocks = (unsigned)std::min<size_t>((count4 + 255) / 256, 152 * 16);
    reduce_splits<<<blocks, 256, 0, st>>>((float4*)final_out, (const float4*)plan->split_buf, a.nsplit, count4);
    count_launch();
    e = cudaGetLastError();
  }
  return cuda_fail(e);
}

// number of partial doubles a reduction over the owners of a mode must sum
int partial_count(hse_plan plan, int mode, int n_own) {
  return plan->nsplit[role_of(mode)] * plan->p.nk * n_own;
}

// Occupied rows of the Fock sum: the caller's arrays, or their sampled rows gathered into
// the plan's compact buffers (down-sampling).
int occupied_rows(hse_plan plan, const void* u_occ, const double* occ, const void** u_rows, const double** occ_rows,
                  cudaStream_t st) {
  if (!plan->sampled) {
    *u_rows = u_occ;
    *occ_rows = occ;
    return HSE_OK;
  }
  const size_t words = (size_t)plan->p.n_occ * plan->N * elem_bytes(plan->p.dtype) / 8;
  const size_t total = words * plan->nkq;
  const unsigned blocks = (unsigned)std::min<size_t>((total + 255) / 256, 152 * 16);
  gather_rows<<<blocks, 256, 0, st>>>((uint64_t*)plan->u_sub, (const uint64_t*)u_occ, plan->d_kocc, plan->nkq, words);
  count_launch();
  gather_rows<<<std::max(1u, (unsigned)((plan->nkq * plan->p.n_occ + 255) / 256)), 256, 0, st>>>(
      (uint64_t*)plan->occ_sub, (const uint64_t*)occ, plan->d_kocc, plan->nkq, (size_t)plan->p.n_occ);
  count_launch();
  *u_rows = plan->u_sub;
  *occ_rows = plan->occ_sub;
  return cuda_fail(cudaGetLastError());
}

// The VJP w.r.t. the sampled occupied orbitals, back on the full mesh (zeros elsewhere).
int scatter_occ_grad(hse_plan plan, void* grad_u_occ, cudaStream_t st) {
  const size_t words = (size_t)plan->p.n_occ * plan->N * elem_bytes(plan->p.dtype) / 8;
  const size_t total = words * plan->p.nk;
  const unsigned blocks = (unsigned)std::min<size_t>((total + 255) / 256, 152 * 16);
  scatter_rows<<<blocks, 256, 0, st>>>((uint64_t*)grad_u_occ, (const uint64_t*)plan->g_sub, plan->d_kinv, plan->p.nk,
                                       words);
  count_launch();
  return cuda_fail(cudaGetLastError());
}

int reduce(hse_plan plan, int n, double factor, double* out, cudaStream_t st, const double* src = nullptr) {
  reduce_partials<<<1, 1024, 0, st>>>(src ? src : plan->partial, n, factor, out);
  count_launch();
  return cuda_fail(cudaGetLastError());
}

// Staged FP64 V_x: out[k][i] for every target; table = v64 or dv64.  u_occ / occ are the
// occupied rows of the Fock sum ([nkq][n_occ]).
int staged_apply(hse_plan plan, const double2* u_occ, const double* occ, const double2* u_tgt, int n_tgt,
                 const double* table, double2* out, cudaStream_t st) {
  const hse_problem& p = plan->p;
  const int N = plan->N;
  const int nk = p.nk, nkq = plan->nkq;
  const size_t per_kp = (size_t)n_tgt * p.n_occ;
  if (per_kp > plan->work_pairs) return HSE_ERR_INVALID_ARG;  // cannot happen: sized for max(n_occ, n_tgt)
  const int nkp_chunk = (int)(plan->work_pairs / per_kp);
  StagedArgs a{};
  a.u_occ = u_occ;
  a.u_tgt = u_tgt;
  a.occ = occ;
  a.vtab = table;
  a.qidx = plan->qidx;
  a.work = plan->work;
  a.nk_occ = nkq;
  a.n_occ = p.n_occ;
  a.n_tgt = n_tgt;
  a.N = N;
  a.scale = -p.alpha / ((double)nkq * N);
  const int inner[3] = {p.grid[1] * p.grid[2], p.grid[2], 1};
  for (int k = 0; k < nk; ++k) {
    for (int kp0 = 0; kp0 < nkq; kp0 += nkp_chunk) {
      a.k = k;
      a.kp0 = kp0;
      a.nkp = std::min(nkp_chunk, nkq - kp0);
      const size_t nb = (size_t)n_tgt * a.nkp * p.n_occ;
      cudaError_t e = launch_staged_pair_product(a, st);
      if (e != cudaSuccess) return cuda_fail(e);
      for (int d = 2; d >= 0; --d) {
        e = launch_staged_fft(p.grid[d], -1, plan->work, nb, N, inner[d], st);
        if (e != cudaSuccess) return cuda_fail(e);
      }
      e = launch_staged_kernel_scale(a, st);
      if (e != cudaSuccess) return cuda_fail(e);
      for (int d = 0; d < 3; ++d) {
        e = launch_staged_fft(p.grid[d], +1, plan->work, nb, N, inner[d], st);
        if (e != cudaSuccess) return cuda_fail(e);
      }
      e = launch_staged_mul_acc(a, out, kp0 == 0, st);
      if (e != cudaSuccess) return cuda_fail(e);
    }
  }
  return HSE_OK;
}

// Work lists of a batched plan for a k' split factor: items (cell, split, k, tile) of the
// sides with a staged-partner pipeline, then those of the pencil-load sides, each sorted by
// cost (partners x grid points x log2 grid points), largest first; sets each cell's split.
void build_batch(hse_plan plan, int split, void* const* vx_out) {
  struct Entry {
    double cost;
    BatchItem it;
  };
  std::vector<Entry> list[3];
  for (size_t c = 0; c < plan->cells.size(); ++c) {
    const hse_problem& q = plan->cells[c]->p;
    BatchCell& bc = plan->h_cells[c];
    const int ns = std::min(split, std::min(kMaxBatchSplit, q.nk));
    bc.pa.nsplit = ns;
    bc.pa.out = ns > 1 ? plan->cell_split[c] : (float2*)vx_out[c];
    const int T = slots_for(q.grid[0]);
    const int ntiles = (q.n_tgt + T - 1) / T;
    const double n = q.grid[0];
    int sp_unused = 0, br_unused = 0;
    // 0: the staged kernel, 1: the pencil-load kernel, 2: the 12^3 LayoutOne kernel
    const int which = !batched_stage_geometry(q.grid[0], &sp_unused, &br_unused) ? 1
                      : (q.grid[0] == 12 && bc.layout == 0)                       ? 2
                                                                                  : 0;
    for (int sp = 0; sp < ns; ++sp) {
      const int kp0 = (int)(((long long)sp * q.nk) / ns), kp1 = (int)(((long long)(sp + 1) * q.nk) / ns);
      const double cost = (double)(kp1 - kp0) * q.n_occ * n * n * n * std::log2(n);
      for (int r = 0; r < q.nk * ntiles; ++r) list[which].push_back({cost, {(int)c, sp * q.nk * ntiles + r}});
    }
  }
  std::vector<BatchItem> items;
  for (int w = 0; w < 3; ++w) {
    std::stable_sort(list[w].begin(), list[w].end(), [](const Entry& x, const Entry& y) { return x.cost > y.cost; });
    for (const Entry& e : list[w]) items.push_back(e.it);
  }
  plan->nitems_staged = (int)list[0].size();
  plan->nitems_pencil = (int)list[1].size();
  plan->nitems = (int)items.size();
  cudaMemcpy(plan->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
}

// The per-cell form of a batched call: each cell's single-cell apply (the kernels and launch
// shape a plan of that cell alone uses) on one of kCellBranches streams forked from st, cells
// in decreasing work, each to the branch with the least work so far.  Graph-capturable once
// every sub-plan's scratch exists (after one uncaptured call).  A failed device-side wait
// records its status in the batched plan's status word.
int run_batch_percell(hse_plan plan, cudaStream_t st) {
  const int ncells = (int)plan->cells.size();
  std::vector<int> order(ncells);
  std::vector<double> cost(ncells);
  for (int c = 0; c < ncells; ++c) {
    const hse_problem& q = plan->cells[c]->p;
    const double n = q.grid[0];
    order[c] = c;
    cost[c] = (double)q.nk * q.n_tgt * q.nk * q.n_occ * n * n * n * std::log2(n);
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  cudaStream_t br[kCellBranches];
  br[0] = st;
  for (int b = 1; b < kCellBranches; ++b) br[b] = plan->cell_side[b - 1];
  cudaError_t e = cudaEventRecord(plan->ev_fork, st);
  for (int b = 1; b < kCellBranches && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(br[b], plan->ev_fork, 0);
  if (e != cudaSuccess) return cuda_fail(e);
  double load[kCellBranches] = {};
  int rc = HSE_OK;
  for (int c : order) {
    int b = 0;
    for (int i = 1; i < kCellBranches; ++i)
      if (load[i] < load[b]) b = i;
    load[b] += cost[c];
    const hse_plan sub = plan->cells[c];
    PairArgs a = base_args(sub);
    a.own = (const float2*)plan->call_ptrs[4 * c + 2];
    a.part = (const float2*)plan->call_ptrs[4 * c + 0];
    a.occ = (const double*)plan->call_ptrs[4 * c + 1];
    a.out = (float2*)plan->call_ptrs[4 * c + 3];
    a.n_part = sub->p.n_occ;
    a.status = plan->status;
    rc = run_pairconv(sub, MODE_APPLY, a, sub->p.n_tgt, br[b]);
    if (rc) break;
  }
  // every branch joins st again, also after an error (no capture is left forked)
  for (int b = 1; b < kCellBranches; ++b) {
    cudaError_t je = cudaEventRecord(plan->cell_join[b - 1], br[b]);
    if (je == cudaSuccess) je = cudaStreamWaitEvent(st, plan->cell_join[b - 1], 0);
    if (je != cudaSuccess && rc == HSE_OK) rc = cuda_fail(je);
  }
  return rc;
}

// counter reset + the two persistent kernels + reduction of split cells (graph-capturable);
// the per-cell form instead when the autotuner chose it
cudaError_t run_batch(hse_plan plan, cudaStream_t st) {
  if (plan->batch_percell) {
    const int rc = run_batch_percell(plan, st);
    if (rc == HSE_OK) plan->percell_warm = true;
    return rc == HSE_OK ? cudaSuccess : (rc == HSE_ERR_NOMEM ? cudaErrorMemoryAllocation : cudaErrorUnknown);
  }
  cudaError_t e = cudaMemsetAsync(plan->d_counter, 0, 3 * sizeof(int), st);
  const int n0 = plan->nitems_staged, n1 = plan->nitems_pencil;
  const BatchArgs staged{plan->d_cells, plan->d_items, n0, plan->d_counter, plan->status};
  const BatchArgs pencil{plan->d_cells, plan->d_items + n0, n1, plan->d_counter + 1, plan->status};
  const BatchArgs staged12{plan->d_cells, plan->d_items + n0 + n1, plan->nitems - n0 - n1, plan->d_counter + 2,
                           plan->status};
  bool pencil_blocked = true;  // every 24^3 cell reads its pencil-blocked copies (set per call)
  for (const BatchCell& bc : plan->h_cells)
    if (bc.n == 24 && bc.pa.blk != 1) pencil_blocked = false;
  if (e == cudaSuccess)
    e = launch_pairconv_batched(staged, staged12, pencil, plan->sms, plan->batch_layout24, pencil_blocked, st,
                                plan->batch_serial ? nullptr : plan->side_stream, plan->ev_fork, plan->ev_join);
  if (e == cudaSuccess && plan->batch_split != 1) {
    reduce_splits_batched<<<plan->sms * 4, 256, 0, st>>>(plan->d_cells, (int)plan->cells.size());
    count_launch();
    e = cudaGetLastError();
  }
  return e;
}

// Staged FP64 VJP: grad_u_tgt = V_x ybar; grad_omega = Re <ybar, V_x' u_tgt> (V_x' with
// d v / d omega rows); grad_u_occ by occupied-owner batches.  u_occ / occ / g_occ are the
// occupied rows of the Fock sum ([nkq][n_occ]).
int staged_vjp(hse_plan plan, const double2* u_occ, const double* occ, const double2* u_tgt, const double2* ybar,
               double2* g_occ, double2* g_tgt, double* g_om, cudaStream_t st) {
  const hse_problem& p = plan->p;
  const int N = plan->N;
  int rc = HSE_OK;
  if (g_tgt) {
    rc = staged_apply(plan, u_occ, occ, ybar, p.n_tgt, plan->v64, g_tgt, st);
    if (rc) return rc;
  }
  if (g_om) {
    rc = staged_apply(plan, u_occ, occ, u_tgt, p.n_tgt, plan->dv64, plan->vx64, st);
    if (rc) return rc;
    dot_per_owner_f64<<<p.nk * p.n_tgt, 256, 0, st>>>(ybar, plan->vx64, N, nullptr, plan->partial);
    count_launch();
    rc = cuda_fail(cudaGetLastError());
    if (rc) return rc;
    rc = reduce(plan, p.nk * p.n_tgt, 1.0, g_om, st);
    if (rc) return rc;
  }
  if (g_occ) {
    // the work buffer holds two pair batches of work_pairs / 2 each
    const size_t per_k = (size_t)p.n_occ * p.n_tgt;
    const size_t half = plan->work_pairs / 2;
    if (per_k > half) return HSE_ERR_NOMEM;
    const int nkc_max = (int)std::min<size_t>(half / per_k, (size_t)p.nk);
    const int nkq = plan->nkq;
    StagedOccArgs a{};
    a.u_occ = u_occ;
    a.u_tgt = u_tgt;
    a.ybar = ybar;
    a.occ = occ;
    a.vtab = plan->v64;
    a.qidx = plan->qidx;
    a.w1 = plan->work;
    a.w2 = plan->work + half * N;
    a.nk_occ = nkq;
    a.n_occ = p.n_occ;
    a.n_tgt = p.n_tgt;
    a.N = N;
    a.scale = -p.alpha / ((double)nkq * N);
    const int inner[3] = {p.grid[1] * p.grid[2], p.grid[2], 1};
    for (int kp = 0; kp < nkq; ++kp) {
      for (int k0 = 0; k0 < p.nk; k0 += nkc_max) {
        a.kp = kp;
        a.k0 = k0;
        a.nkc = std::min(nkc_max, p.nk - k0);
        const size_t nb = per_k * a.nkc;
        cudaError_t e = launch_staged_occ_products(a, st);
        for (int d = 2; d >= 0 && e == cudaSuccess; --d) {
          e = launch_staged_fft(p.grid[d], -1, a.w1, nb, N, inner[d], st);
          if (e == cudaSuccess) e = launch_staged_fft(p.grid[d], -1, a.w2, nb, N, inner[d], st);
        }
        if (e == cudaSuccess) e = launch_staged_occ_scale(a, st);
        for (int d = 0; d < 3 && e == cudaSuccess; ++d) {
          e = launch_staged_fft(p.grid[d], +1, a.w1, nb, N, inner[d], st);
          if (e == cudaSuccess) e = launch_staged_fft(p.grid[d], +1, a.w2, nb, N, inner[d], st);
        }
        if (e == cudaSuccess) e = launch_staged_occ_acc(a, g_occ, k0 == 0, st);
        if (e != cudaSuccess) return cuda_fail(e);
      }
    }
  }
  return rc;
}

}  // namespace

extern "C" {

int hse_fock_apply(hse_plan plan, const void* u_occ, const double* occ, const void* u_tgt, void* vx_out,
                   hse_stream_t stream) {
  const NvtxRange nvtx_range("hse_fock_apply");
  if (!plan || !u_occ || !occ || !u_tgt || !vx_out) return HSE_ERR_INVALID_ARG;
  const hse_problem& p = plan->p;
  if (!aligned16(u_occ) || !aligned16(u_tgt) || !aligned16(vx_out)) return HSE_ERR_INVALID_ARG;
  const size_t eb = elem_bytes(p.dtype);
  const size_t occ_bytes = (size_t)p.nk * p.n_occ * plan->N * eb;
  const size_t tgt_bytes = (size_t)p.nk * p.n_tgt * plan->N * eb;
  if (overlaps(vx_out, tgt_bytes, u_occ, occ_bytes) || overlaps(vx_out, tgt_bytes, u_tgt, tgt_bytes) ||
      overlaps(vx_out, tgt_bytes, occ, (size_t)p.nk * p.n_occ * sizeof(double)))
    return HSE_ERR_ALIAS;
  cudaStream_t st = S(stream);
  const void* u_rows = nullptr;
  const double* occ_rows = nullptr;
  int rc = occupied_rows(plan, u_occ, occ, &u_rows, &occ_rows, st);
  if (rc) return rc;
  if (p.dtype == HSE_C64) {
    PairArgs a = base_args(plan);
    a.own = (const float2*)u_tgt;
    a.part = (const float2*)u_rows;
    a.out = (float2*)vx_out;
    a.occ = occ_rows;
    a.n_part = p.n_occ;
    return run_pairconv(plan, MODE_APPLY, a, p.n_tgt, st);
  }
  return staged_apply(plan, (const double2*)u_rows, occ_rows, (const double2*)u_tgt, p.n_tgt, plan->v64,
                      (double2*)vx_out, st);
}

int hse_exchange_energy(hse_plan plan, const void* u_occ, const double* occ, double* e_x, hse_stream_t stream) {
  const NvtxRange nvtx_range("hse_exchange_energy");
  if (!plan || !u_occ || !occ || !e_x) return HSE_ERR_INVALID_ARG;
  const hse_problem& p = plan->p;
  if (!aligned16(u_occ)) return HSE_ERR_INVALID_ARG;
  cudaStream_t st = S(stream);
  const int nown = p.nk * p.n_occ;
  const double factor = 0.5 * p.spin_degeneracy * plan->dV / p.nk;
  // targets: the occupied orbitals at every k-point; partners: the rows of the Fock sum
  const void* u_rows = nullptr;
  const double* occ_rows = nullptr;
  int rc = occupied_rows(plan, u_occ, occ, &u_rows, &occ_rows, st);
  if (rc) return rc;
  if (p.dtype == HSE_C64) {
    PairArgs a = base_args(plan);
    a.own = (const float2*)u_occ;
    a.part = (const float2*)u_rows;
    a.partial = plan->partial;
    a.occ = occ_rows;
    a.occ_own = occ;
    a.n_part = p.n_occ;
    rc = run_pairconv(plan, MODE_ENERGY, a, p.n_occ, st);
  } else {
    rc = staged_apply(plan, (const double2*)u_rows, occ_rows, (const double2*)u_occ, p.n_occ, plan->v64, plan->vx64,
                      st);
    if (rc) return rc;
    dot_per_owner_f64<<<nown, 256, 0, st>>>((const double2*)u_occ, plan->vx64, plan->N, occ, plan->partial);
    count_launch();
    rc = cuda_fail(cudaGetLastError());
  }
  if (rc) return rc;
  return reduce(plan, p.dtype == HSE_C64 ? partial_count(plan, MODE_ENERGY, p.n_occ) : nown, factor, e_x, st);
}

int hse_fock_apply_vjp(hse_plan plan, const void* u_occ, const double* occ, const void* u_tgt, const void* grad_vx,
                       void* grad_u_occ, void* grad_u_tgt, double* grad_omega, hse_stream_t stream) {
  const NvtxRange nvtx_range("hse_fock_apply_vjp");
  if (!plan || !u_occ || !occ || !u_tgt || !grad_vx) return HSE_ERR_INVALID_ARG;
  const hse_problem& p = plan->p;
  if (!aligned16(u_occ) || !aligned16(u_tgt) || !aligned16(grad_vx) || (grad_u_occ && !aligned16(grad_u_occ)) ||
      (grad_u_tgt && !aligned16(grad_u_tgt)))
    return HSE_ERR_INVALID_ARG;
  const size_t eb = elem_bytes(p.dtype);
  const size_t occ_bytes = (size_t)p.nk * p.n_occ * plan->N * eb;
  const size_t tgt_bytes = (size_t)p.nk * p.n_tgt * plan->N * eb;
  const void* ins[4] = {u_occ, u_tgt, grad_vx, occ};
  const size_t insz[4] = {occ_bytes, tgt_bytes, tgt_bytes, (size_t)p.nk * p.n_occ * sizeof(double)};
  for (int i = 0; i < 4; ++i) {
    if (overlaps(grad_u_occ, occ_bytes, ins[i], insz[i]) || overlaps(grad_u_tgt, tgt_bytes, ins[i], insz[i]) ||
        overlaps(grad_omega, sizeof(double), ins[i], insz[i]))
      return HSE_ERR_ALIAS;
  }
  if (overlaps(grad_u_occ, occ_bytes, grad_u_tgt, tgt_bytes)) return HSE_ERR_ALIAS;
  cudaStream_t st = S(stream);
  const void* u_rows = nullptr;
  const double* occ_rows = nullptr;
  int rc = occupied_rows(plan, u_occ, occ, &u_rows, &occ_rows, st);
  if (rc) return rc;
  // the VJP w.r.t. the sampled rows goes to the plan's compact buffer, then to the full mesh
  void* g_rows = (grad_u_occ && plan->sampled) ? plan->g_sub : grad_u_occ;
  if (p.dtype == HSE_C128) {
    rc = staged_vjp(plan, (const double2*)u_rows, occ_rows, (const double2*)u_tgt, (const double2*)grad_vx,
                    (double2*)g_rows, (double2*)grad_u_tgt, grad_omega, st);
    if (rc == HSE_OK && grad_u_occ && plan->sampled) rc = scatter_occ_grad(plan, grad_u_occ, st);
    return rc;
  }
  if (grad_u_tgt) {
    PairArgs a = base_args(plan);
    a.own = (const float2*)grad_vx;
    a.part = (const float2*)u_rows;
    a.out = (float2*)grad_u_tgt;
    a.occ = occ_rows;
    a.n_part = p.n_occ;
    rc = run_pairconv(plan, MODE_APPLY, a, p.n_tgt, st);
    if (rc) return rc;
  }
  // with both, the omega gradient rides on the u_occ pass's transforms (Parseval); alone it
  // takes a pass of its own
  const bool fuse_w = grad_omega && grad_u_occ;
  if (grad_omega && !fuse_w) {
    PairArgs a = base_args(plan);
    a.own = (const float2*)u_tgt;
    a.part = (const float2*)u_rows;
    a.part2 = (const float2*)grad_vx;
    a.partial = plan->partial;
    a.occ = occ_rows;
    a.vtab = plan->dv32;
    a.n_part = p.n_occ;
    rc = run_pairconv(plan, MODE_DOT, a, p.n_tgt, st);
    if (rc) return rc;
    rc = reduce(plan, partial_count(plan, MODE_DOT, p.n_tgt), 1.0, grad_omega, st);
    if (rc) return rc;
  }
  if (grad_u_occ) {
    // owners: the occupied orbitals of the Fock sum (nkq k-points); partners: all targets
    PairArgs a = base_args(plan);
    a.own = (const float2*)u_rows;
    a.part = (const float2*)u_tgt;
    a.part2 = (const float2*)grad_vx;
    a.out = (float2*)g_rows;
    a.occ = occ_rows;
    a.nk_own = plan->nkq;
    a.nk_part = p.nk;
    a.n_part = p.n_tgt;
    if (fuse_w) a.vtab2 = plan->dv32;
    rc = run_pairconv(plan, MODE_OCC, a, p.n_occ, st);
    if (rc == HSE_OK && fuse_w) {
      const int T = slots_for(p.grid[0]);
      const int items = plan->nsplit[ROLE_OCC] * plan->nkq * ((p.n_occ + T - 1) / T);
      rc = reduce(plan, items, 1.0, grad_omega, st, plan->wpartial);
    }
    if (rc == HSE_OK && plan->sampled) rc = scatter_occ_grad(plan, grad_u_occ, st);
  }
  return rc;
}

int hse_kinetic_apply(hse_plan plan, const void* u, int nbands, const double* A, void* out, hse_stream_t stream) {
  const NvtxRange nvtx_range("hse_kinetic_apply");
  if (!plan || !u || !out || !A || nbands < 1) return HSE_ERR_INVALID_ARG;
  for (int c = 0; c < 3; ++c)
    if (!std::isfinite(A[c])) return HSE_ERR_INVALID_ARG;
  if (!aligned16(u) || !aligned16(out)) return HSE_ERR_INVALID_ARG;
  const hse_problem& p = plan->p;
  const size_t bytes = (size_t)p.nk * nbands * plan->N * elem_bytes(p.dtype);
  if (overlaps(out, bytes, u, bytes)) return HSE_ERR_ALIAS;
  KinArgs a{};
  a.n1 = p.grid[0];
  a.n2 = p.grid[1];
  a.n3 = p.grid[2];
  a.nk = p.nk;
  a.nbands = nbands;
  std::memcpy(a.b, plan->b, sizeof(a.b));
  for (int c = 0; c < 3; ++c) a.A[c] = A[c];
  a.kpts = plan->dkpts;
  cudaStream_t st = S(stream);
  if (p.dtype == HSE_C64) {
    const int T = slots_for(p.grid[0]);
    a.ntiles = (nbands + T - 1) / T;
    return cuda_fail(launch_kinetic_c64(p.grid[0], (const float2*)u, (float2*)out, a, st));
  }
  return cuda_fail(launch_kinetic_f64((const double2*)u, (double2*)out, a, st));
}

int hse_taylor_step(hse_plan plan, const void* psi, const double* occ, const double* A, double dt, const double* vloc,
                    void* psi_out, hse_stream_t stream) {
  const NvtxRange nvtx_range("hse_taylor_step");
  if (!plan || plan->batched || !psi || !occ || !A || !psi_out || !std::isfinite(dt)) return HSE_ERR_INVALID_ARG;
  const hse_problem& p = plan->p;
  if (p.n_tgt != p.n_occ) return HSE_ERR_INVALID_ARG;  // the step propagates the occupied set
  for (int c = 0; c < 3; ++c)
    if (!std::isfinite(A[c])) return HSE_ERR_INVALID_ARG;
  if (!aligned16(psi) || !aligned16(psi_out)) return HSE_ERR_INVALID_ARG;
  const size_t count = (size_t)p.nk * p.n_occ * plan->N;
  const size_t bytes = count * elem_bytes(p.dtype);
  if (overlaps(psi_out, bytes, psi, bytes) || overlaps(psi_out, bytes, occ, (size_t)p.nk * p.n_occ * sizeof(double)) ||
      overlaps(psi_out, bytes, vloc, (size_t)plan->N * sizeof(double)))
    return HSE_ERR_ALIAS;
  for (void*& b : plan->tay)
    if (!b) {
      const cudaError_t e = plan_malloc(plan, &b, bytes);
      if (e != cudaSuccess) return cuda_fail(e);
    }
  cudaStream_t st = S(stream);
  cudaError_t e = cudaMemcpyAsync(psi_out, psi, bytes, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e);
  const void* term = psi;
  for (int n = 1; n <= 4; ++n) {
    int rc = hse_kinetic_apply(plan, term, p.n_occ, A, plan->tay[1], stream);
    if (rc) return rc;
    rc = hse_fock_apply(plan, psi, occ, term, plan->tay[2], stream);
    if (rc) return rc;
    e = launch_taylor_accumulate(p.dtype == HSE_C128, plan->tay[1], plan->tay[2], term, vloc, (size_t)plan->N,
                                 plan->tay[0], psi_out, count, dt / n, st);
    if (e != cudaSuccess) return cuda_fail(e);
    term = plan->tay[0];
  }
  return HSE_OK;
}

int hse_current(hse_plan plan, const void* psi, const double* occ, const double* A, double* J, hse_stream_t stream) {
  const NvtxRange nvtx_range("hse_current");
  if (!plan || plan->batched || !psi || !occ || !A || !J) return HSE_ERR_INVALID_ARG;
  for (int c = 0; c < 3; ++c)
    if (!std::isfinite(A[c])) return HSE_ERR_INVALID_ARG;
  if (!aligned16(psi)) return HSE_ERR_INVALID_ARG;
  const hse_problem& p = plan->p;
  const size_t norb = (size_t)p.nk * p.n_occ;
  if (!plan->cur_work) {
    cudaError_t e = plan_malloc(plan, &plan->cur_work, norb * plan->N * sizeof(double2));
    if (e == cudaSuccess) e = plan_malloc(plan, &plan->cur_partial, norb * 3 * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(e);
  }
  CurArgs a{};
  a.n1 = p.grid[0];
  a.n2 = p.grid[1];
  a.n3 = p.grid[2];
  a.nk = p.nk;
  a.nbands = p.n_occ;
  std::memcpy(a.b, plan->b, sizeof(a.b));
  for (int c = 0; c < 3; ++c) a.A[c] = A[c];
  a.kpts = plan->dkpts;
  return cuda_fail(launch_current(p.dtype == HSE_C128, psi, occ, a, plan->cur_work, plan->cur_partial,
                                  p.spin_degeneracy, J, S(stream)));
}

int hse_overlap(hse_plan plan, const void* u, int nbands, double* s_out, hse_stream_t stream) {
  const NvtxRange nvtx_range("hse_overlap");
  if (!plan || plan->batched || !u || !s_out || nbands < 1 || nbands > 4096 || plan->p.nk > 65535)
    return HSE_ERR_INVALID_ARG;
  if (!aligned16(u) || !aligned16(s_out)) return HSE_ERR_INVALID_ARG;
  const hse_problem& p = plan->p;
  const size_t ub = (size_t)p.nk * nbands * plan->N * elem_bytes(p.dtype);
  if (overlaps(s_out, (size_t)p.nk * nbands * nbands * 2 * sizeof(double), u, ub)) return HSE_ERR_ALIAS;
  return cuda_fail(launch_overlap(p.dtype == HSE_C128, u, p.nk, nbands, plan->N, plan->dV, (double2*)s_out, S(stream)));
}

int hse_orthonormalize(hse_plan plan, void* u, int nbands, hse_stream_t stream) {
  const NvtxRange nvtx_range("hse_orthonormalize");
  if (!plan || plan->batched || !u || nbands < 1 || nbands > 4096) return HSE_ERR_INVALID_ARG;
  if (!aligned16(u)) return HSE_ERR_INVALID_ARG;
  const hse_problem& p = plan->p;
  const size_t count = (size_t)p.nk * nbands * plan->N;
  if (p.dtype == HSE_C64 && count > plan->ortho_elems) {
    cudaFree(plan->ortho_work);
    plan->ortho_work = nullptr;
    plan->ortho_elems = 0;
    const cudaError_t e = plan_malloc(plan, &plan->ortho_work, count * sizeof(double2));
    if (e != cudaSuccess) return cuda_fail(e);
    plan->ortho_elems = count;
  }
  return cuda_fail(launch_orthonormalize(p.dtype == HSE_C128, u, p.nk, nbands, plan->N, plan->dV, plan->ortho_work,
                                         plan->status, S(stream)));
}

int hse_hartree_potential(hse_plan plan, const void* psi, const double* occ, double* vh, hse_stream_t stream) {
  const NvtxRange nvtx_range("hse_hartree_potential");
  if (!plan || plan->batched || !psi || !occ || !vh) return HSE_ERR_INVALID_ARG;
  if (!aligned16(psi)) return HSE_ERR_INVALID_ARG;
  const hse_problem& p = plan->p;
  if (!plan->hart_work) {
    const cudaError_t e = plan_malloc(plan, &plan->hart_work, (size_t)plan->N * sizeof(double2));
    if (e != cudaSuccess) return cuda_fail(e);
  }
  CurArgs a{};
  a.n1 = p.grid[0];
  a.n2 = p.grid[1];
  a.n3 = p.grid[2];
  a.nk = p.nk;
  a.nbands = p.n_occ;
  std::memcpy(a.b, plan->b, sizeof(a.b));
  a.kpts = plan->dkpts;
  return cuda_fail(launch_hartree(p.dtype == HSE_C128, psi, occ, a, p.spin_degeneracy, plan->hart_work, vh, S(stream)));
}

int hse_plan_create_batched(hse_plan* out, const hse_problem* cells, int ncells) {
  const NvtxRange nvtx_range("hse_plan_create_batched");
  if (!out) return HSE_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cells || ncells < 1 || ncells > 65536) return HSE_ERR_INVALID_ARG;
  for (int c = 0; c < ncells; ++c) {
    const int rc = validate_problem(&cells[c]);
    if (rc) return rc;
    if (cells[c].dtype != HSE_C64 || !batched_side_supported(cells[c].grid[0])) return HSE_ERR_UNSUPPORTED_GRID;
    if (cells[c].nk_occ != 0) return HSE_ERR_INVALID_ARG;  // down-sampling: single-cell plans only
  }
  hse_plan plan = new (std::nothrow) hse_plan_s();
  if (!plan) return HSE_ERR_NOMEM;
  plan->batched = true;
  plan->fail_alloc_at = fail_alloc_from_env();
  plan->p = cells[0];
  cudaGetDevice(&plan->device);
  int rc = HSE_OK;
  cudaError_t e = cudaDeviceGetAttribute(&plan->sms, cudaDevAttrMultiProcessorCount, plan->device);
  size_t max_items = 0;
  for (int c = 0; c < ncells && rc == HSE_OK && e == cudaSuccess; ++c) {
    hse_plan sub = nullptr;
    rc = hse_plan_create(&sub, &cells[c]);
    if (rc) break;
    plan->cells.push_back(sub);
    const hse_problem& q = sub->p;
    const int T = slots_for(q.grid[0]);
    const int ntiles = (q.n_tgt + T - 1) / T;
    max_items += (size_t)std::min(kMaxBatchSplit, q.nk) * q.nk * ntiles;
    float2* buf = nullptr;
    if (q.nk > 1) e = plan_malloc(plan, &buf, (size_t)std::min(kMaxBatchSplit, q.nk) * q.nk * q.n_tgt * sub->N * sizeof(float2));
    plan->cell_split.push_back(buf);
    float2* comp = nullptr;
    if (e == cudaSuccess)
      e = plan_malloc(plan, &comp, (size_t)std::min(kMaxBatchSplit, q.nk) * q.nk * q.n_tgt * 2 * blocked_stride(q.grid[0]) *
                                sizeof(float2));
    plan->cell_comp.push_back(comp);
    float2* blk = nullptr;
    int sp = 0, br = 0;
    if (e == cudaSuccess && !batched_stage_geometry(q.grid[0], &sp, &br))
      e = plan_malloc(plan, &blk, (size_t)q.nk * (q.n_tgt + q.n_occ) * blocked_stride(q.grid[0]) * sizeof(float2));
    plan->cell_blk.push_back(blk);
  }
  if (rc == HSE_OK && e == cudaSuccess) e = plan_malloc(plan, &plan->d_cells, (size_t)ncells * sizeof(BatchCell));
  if (rc == HSE_OK && e == cudaSuccess) e = plan_malloc(plan, &plan->d_items, max_items * sizeof(BatchItem));
  if (rc == HSE_OK && e == cudaSuccess) e = plan_malloc(plan, &plan->d_counter, 3 * sizeof(int));
  if (rc == HSE_OK && e == cudaSuccess) e = plan_malloc(plan, &plan->status, sizeof(int));
  if (rc == HSE_OK && e == cudaSuccess) e = cudaMemset(plan->status, 0, sizeof(int));
  if (rc == HSE_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(&plan->capture_stream, cudaStreamNonBlocking);
  if (rc == HSE_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(&plan->side_stream, cudaStreamNonBlocking);
  if (rc == HSE_OK && e == cudaSuccess) e = cudaEventCreateWithFlags(&plan->ev_fork, cudaEventDisableTiming);
  if (rc == HSE_OK && e == cudaSuccess) e = cudaEventCreateWithFlags(&plan->ev_join, cudaEventDisableTiming);
  for (int b = 0; b < kCellBranches - 1; ++b) {
    if (rc == HSE_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(&plan->cell_side[b], cudaStreamNonBlocking);
    if (rc == HSE_OK && e == cudaSuccess) e = cudaEventCreateWithFlags(&plan->cell_join[b], cudaEventDisableTiming);
  }
  if (rc == HSE_OK && e != cudaSuccess) rc = cuda_fail(e);
  if (rc) {
    hse_plan_destroy(plan);
    return rc;
  }
  plan->h_cells.resize(ncells);
  *out = plan;
  return HSE_OK;
}

int hse_fock_apply_batched(hse_plan plan, const void* const* u_occ, const double* const* occ, const void* const* u_tgt,
                           void* const* vx_out, hse_stream_t stream) {
  const NvtxRange nvtx_range("hse_fock_apply_batched");
  if (!plan || !plan->batched || !u_occ || !occ || !u_tgt || !vx_out) return HSE_ERR_INVALID_ARG;
  const int ncells = (int)plan->cells.size();
  for (int c = 0; c < ncells; ++c) {
    const hse_plan sub = plan->cells[c];
    const hse_problem& q = sub->p;
    if (!u_occ[c] || !occ[c] || !u_tgt[c] || !vx_out[c]) return HSE_ERR_INVALID_ARG;
    if (!aligned16(u_occ[c]) || !aligned16(u_tgt[c]) || !aligned16(vx_out[c])) return HSE_ERR_INVALID_ARG;
    const size_t ob = (size_t)q.nk * q.n_occ * sub->N * 8, tb = (size_t)q.nk * q.n_tgt * sub->N * 8;
    if (overlaps(vx_out[c], tb, u_occ[c], ob) || overlaps(vx_out[c], tb, u_tgt[c], tb) ||
        overlaps(vx_out[c], tb, occ[c], (size_t)q.nk * q.n_occ * sizeof(double)))
      return HSE_ERR_ALIAS;
    for (int d = 0; d < c; ++d) {
      const hse_problem& r = plan->cells[d]->p;
      if (overlaps(vx_out[c], tb, vx_out[d], (size_t)r.nk * r.n_tgt * plan->cells[d]->N * 8)) return HSE_ERR_ALIAS;
    }
  }
  cudaStream_t st = S(stream);
  plan->call_ptrs.resize(4 * (size_t)ncells);
  for (int c = 0; c < ncells; ++c) {
    plan->call_ptrs[4 * c + 0] = u_occ[c];
    plan->call_ptrs[4 * c + 1] = occ[c];
    plan->call_ptrs[4 * c + 2] = u_tgt[c];
    plan->call_ptrs[4 * c + 3] = vx_out[c];
  }
  // per-call pointers into the cell table; the split structure is set by build_batch
  for (int c = 0; c < ncells; ++c) {
    BatchCell& bc = plan->h_cells[c];
    const hse_plan sub = plan->cells[c];
    PairArgs a = base_args(sub);
    a.own = (const float2*)u_tgt[c];
    a.part = (const float2*)u_occ[c];
    a.occ = occ[c];
    a.n_part = sub->p.n_occ;
    a.n_own = sub->p.n_tgt;
    const int T = slots_for(sub->p.grid[0]);
    a.ntiles = (a.n_own + T - 1) / T;
    a.status = plan->status;
    a.nsplit = bc.pa.nsplit > 0 ? bc.pa.nsplit : 1;
    a.split_stride = (size_t)sub->p.nk * a.n_own * sub->N;
    a.out = a.nsplit > 1 ? plan->cell_split[c] : (float2*)vx_out[c];
    a.comp = plan->cell_comp[c];
    if (plan->cell_blk[c]) {
      // the pencil-load pipeline reads pencil-blocked copies (refreshed on every call, before
      // the graph)
      const int n = sub->p.grid[0];
      const size_t nbk = blocked_stride(n);
      const size_t ntgt = (size_t)sub->p.nk * sub->p.n_tgt, nocc = (size_t)sub->p.nk * sub->p.n_occ;
      float2* bt = plan->cell_blk[c];
      float2* bo = bt + ntgt * nbk;
      const float2* srcs[2] = {a.own, a.part};
      float2* dsts[2] = {bt, bo};
      const size_t norbs[2] = {ntgt, nocc};
      for (int i = 0; i < 2; ++i) {
        if (i == 1 && srcs[1] == srcs[0] && nocc == ntgt) {
          dsts[1] = bt;
          break;
        }
        const size_t count4 = norbs[i] * sub->N / 2;
        const unsigned blocks = (unsigned)std::min<size_t>((count4 + 255) / 256, 152 * 16);
        to_pencil_blocks<<<blocks, 256, 0, st>>>((float4*)dsts[i], (const float4*)srcs[i], n, nbk / 2, norbs[i]);
        count_launch();
      }
      a.own = dsts[0];
      a.part = dsts[1];
      a.blk = 1;
      const cudaError_t le = cudaGetLastError();
      if (le != cudaSuccess) return cuda_fail(le);
    }
    bc.pa = a;
    bc.final_out = (float2*)vx_out[c];
    bc.n = sub->p.grid[0];
    int sp = 0, br = 0;
    if (batched_stage_geometry(bc.n, &sp, &br)) {
      const cudaError_t te = make_partner_tmap(&bc.tmap, u_occ[c], bc.n,
                                               (long long)sub->p.nk * sub->p.n_occ * bc.n * bc.n, sp, br);
      if (te != cudaSuccess) return cuda_fail(te);
    } else {
      std::memset(&bc.tmap, 0, sizeof(bc.tmap));
    }
  }
  cudaError_t e = cudaSuccess;
  if (plan->batch_split == 0) {
    // Autotune the shape of the launch on this first call, unless the autotune cache
    // (HSE_AUTOTUNE_CACHE) already holds a choice for this GPU and cell list: the k'-split
    // granularity of the work items, the pencil layout of the 24^3 items, the pencil layout of
    // each staged side, and whether the two persistent kernels run at once.  Coordinate
    // descent from the defaults, each candidate timed on the real inputs.
    const std::string key = autotune_key(plan);
    const int cached = autotune_lookup(key);
    bool has24 = false, present[kShapeSides] = {false, false, false, false, false};
    int nstaged_cells = 0;
    for (hse_plan c : plan->cells) {
      const int n = c->p.grid[0];
      has24 = has24 || n == 24;
      if (side_slot(n) >= 0) present[side_slot(n)] = true;
      if (n != 24) ++nstaged_cells;
    }
    auto apply = [&](const BatchShape& s) {
      plan->batch_percell = s.percell;
      plan->batch_layout24 = s.layout24;
      plan->batch_serial = s.serial;
      for (int c = 0; c < ncells; ++c) {
        const int slot = side_slot(plan->h_cells[c].n);
        plan->h_cells[c].layout = slot >= 0 ? s.seq[slot] : 0;
      }
      build_batch(plan, s.split, vx_out);  // the lists depend on the layouts
    };
    BatchShape best = cached > 0 ? BatchShape::decode(cached) : BatchShape();
    if (cached <= 0) {
      cudaEvent_t t0 = nullptr, t1 = nullptr;
      e = cudaEventCreate(&t0);
      if (e == cudaSuccess) e = cudaEventCreate(&t1);
      auto time_shape = [&](const BatchShape& s, float* ms) {
        apply(s);
        cudaError_t r = cudaMemcpyAsync(plan->d_cells, plan->h_cells.data(), ncells * sizeof(BatchCell),
                                        cudaMemcpyHostToDevice, st);
        if (r == cudaSuccess) r = cudaEventRecord(t0, st);
        if (r == cudaSuccess) r = run_batch(plan, st);
        if (r == cudaSuccess) r = cudaEventRecord(t1, st);
        if (r == cudaSuccess) r = cudaEventSynchronize(t1);
        if (r == cudaSuccess) r = cudaEventElapsedTime(ms, t0, t1);
        if (r == cudaSuccess && log_on()) {
          if (s.percell)
            std::fprintf(stderr, "hse: batched autotune: shape %d (per-cell launches on %d branches): %.3f ms\n",
                         s.encode(), kCellBranches, *ms);
          else
            std::fprintf(stderr,
                         "hse: batched autotune: shape %d (k' split %d, 24^3 %s, %s, LayoutSeq at 8 16 18 20 12: "
                         "%d %d %d %d %d): %.3f ms\n",
                         s.encode(), s.split, s.layout24 == kPencilRagged ? "ragged" : "one pencil",
                         s.serial ? "serial" : "concurrent", s.seq[0], s.seq[1], s.seq[2], s.seq[3], s.seq[4], *ms);
        }
        return r;
      };
      float best_ms = 0.f;
      if (e == cudaSuccess) e = time_shape(best, &best_ms);
      auto trial = [&](const BatchShape& s) {
        float ms = 0.f;
        if (e == cudaSuccess) e = time_shape(s, &ms);
        if (e == cudaSuccess && ms < best_ms) {
          best = s;
          best_ms = ms;
        }
      };
      const BatchShape base = best;
      for (int split : {2, 4}) {
        BatchShape s = base;
        s.split = split;
        trial(s);
      }
      if (has24) {
        BatchShape s = best;
        s.layout24 = kPencilRagged;
        trial(s);
      }
      for (int i = 0; i < kShapeSides; ++i) {
        if (!present[i]) continue;
        BatchShape s = best;
        s.seq[i] = 1;
        trial(s);
      }
      if (has24 && nstaged_cells > 0) {
        BatchShape s = best;
        s.serial = true;
        trial(s);
      }
      {
        BatchShape s;  // the per-cell form (its other fields are unused)
        s.percell = true;
        trial(s);
      }
      if (t0) cudaEventDestroy(t0);
      if (t1) cudaEventDestroy(t1);
      if (e != cudaSuccess) return cuda_fail(e);
      autotune_store(key, best.encode());
    } else if (log_on()) {
      std::fprintf(stderr, "hse: batched autotune: shape %d from the cache\n", cached);
    }
    plan->batch_split = best.split;
    if (log_on()) std::fprintf(stderr, "hse: batched autotune: chose shape %d\n", best.encode());
    apply(best);
  }
  // Capture counter reset + persistent kernels + split reduction (or the per-cell launches) as
  // one graph.  The persistent form reads this call's pointers from the cell table, so its graph
  // serves every later call; the per-cell form's kernels take them as launch arguments, so it is
  // captured again when a call passes other arrays.
  if (!plan->graph || (plan->batch_percell && plan->call_ptrs != plan->graph_ptrs)) {
    if (plan->batch_percell && !plan->percell_warm) {  // the sub-plans allocate scratch on first use
      e = run_batch(plan, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    if (plan->graph) {
      cudaGraphExecDestroy(plan->graph);
      plan->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(plan->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t er = run_batch(plan, plan->capture_stream);
      e = cudaStreamEndCapture(plan->capture_stream, &g);
      if (e == cudaSuccess) e = er;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e);
    plan->graph_ptrs = plan->call_ptrs;
  }
  e = cudaMemcpyAsync(plan->d_cells, plan->h_cells.data(), ncells * sizeof(BatchCell), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaGraphLaunch(plan->graph, st);
  return cuda_fail(e);
}

}  // extern "C"
