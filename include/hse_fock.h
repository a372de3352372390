/*
 * hse_fock.h - C ABI of the GB300 (sm_103a) HSE short-range Fock-like exchange library.
 *
 * The operation is the nonlocal Fock-like term of the HSE exchange-correlation
 * potential of Sato, Taniguchi, Shinohara & Yabana, arXiv:1507.05156:
 *   Sec. II B   - HSE v_xc = v_xc^PBE - 1/4 v_x^{SR,PBE} + 1/4 v^{SR,Fock}, range
 *                 separation mu (called omega here);
 *   Sec. II C   - the real-space definition of v^{SR,Fock} psi_i, its Fourier-space
 *                 form (Eq. "Fock": pair density -> FFT -> kernel -> inverse FFT ->
 *                 multiply by psi_j -> sum over occupied j) and the k/band form
 *                 (Eq. "Fock-DS");
 *   Sec. V      - the exchange-correlation energy E_xc in the excitation energy
 *                 (Eq. "Eex01"), whose Fock part hse_exchange_energy returns.
 *
 * With u_{b,k} the periodic parts of the Bloch orbitals (cell-normalised,
 * dV sum_r |u|^2 = 1, dV = Omega/N), q = k - k' (not folded), and the short-range
 * kernel v(g) = 4 pi / g^2 (1 - exp(-g^2 / 4 omega^2)), v(0) = pi / omega^2:
 *
 *   (V_x u)_{i,k}(r) = -alpha (1/N_k) sum_{k'} sum_{j occ} f_{j,k'} u_{j,k'}(r)
 *                      sum_G v(|G+q|) rho~_{ji}(G) e^{iG.r},
 *   rho~_{ji}(G)     = (1/N) sum_r conj(u_{j,k'}(r)) u_{i,k}(r) e^{-iG.r}.
 * With down-sampling (hse_problem.nk_occ > 0) k' runs over the sampled points and 1/N_k
 * becomes 1/nk_occ in V_x (and in c_j below); E_x keeps 1/N_k over its target k-points.
 *
 * Data layout (all device arrays are caller-owned):
 *   orbitals      [nk][nbands][N1][N2][N3], C order, N3 fastest, interleaved complex:
 *                 float2 (complex64) for HSE_C64, double2 (complex128) for HSE_C128.
 *   occupations   [nk][n_occ] double, f in [0, 1] per spin-orbital.
 *   grid point (i1,i2,i3) is r = i1/N1 a1 + i2/N2 a2 + i3/N3 a3; G = m1 b1 + m2 b2 + m3 b3
 *   with m_d in FFT order (0..ceil(N/2)-1, then -floor(N/2)..-1).
 *
 * Calls are asynchronous on the caller's stream (a cudaStream_t passed as void*,
 * NULL = legacy default stream) and return an hse error code; device-side failures
 * are reported by hse_status.  The library never frees caller memory.  It allocates
 * only its plan (kernel tables and reduction scratch) in hse_plan_create*.
 */
#ifndef HSE_FOCK_H
#define HSE_FOCK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes: 0 is success, every failure is negative. */
#define HSE_OK                    0
#define HSE_ERR_INVALID_ARG      -1  /* null pointer, bad size, bad parameter            */
#define HSE_ERR_UNSUPPORTED_GRID -2  /* an axis length this build has no kernel for     */
#define HSE_ERR_ALIAS            -3  /* an output buffer overlaps an input              */
#define HSE_ERR_CUDA             -4  /* a CUDA runtime call failed                      */
#define HSE_ERR_TIMEOUT          -5  /* a bounded device-side wait gave up              */
#define HSE_ERR_NOMEM            -6  /* plan allocation failed                          */
#define HSE_ERR_DEVICE           -7  /* a kernel recorded a failed device-side check    */
#define HSE_ERR_SINGULAR         -8  /* orthonormalisation met a linearly dependent band */

/* Arithmetic of the pair convolutions. */
#define HSE_C64   0  /* complex64 orbitals, fused FP32 kernel, FP64 energy/omega reduction */
#define HSE_C128  1  /* complex128 orbitals, plain staged FP64 kernels                     */
/* complex64 orbitals (as HSE_C64), the Y and X axis transforms of V_x u and E_x as split-FP16
 * tensor-core GEMMs (hi/lo halves, three products, FP32 accumulation), the Z transforms and
 * every other step as HSE_C64; 24^3 grids only (else HSE_ERR_UNSUPPORTED_GRID).  The VJP's
 * u_occ pass runs the FP32 kernel.  Errors against FP64 stay within 1e-5 but are larger than
 * HSE_C64's, and the FP32 kernel is faster on GB300; an option for study. */
#define HSE_C64_TC 2

typedef void *hse_stream_t;  /* a cudaStream_t */

/* One exchange problem (Sec. II C): a cell, its k-mesh and its band counts. */
typedef struct {
  int grid[3];            /* N1, N2, N3; every axis a product of 2, 3, 5 from the supported set
                             (hse_grid_supported); HSE_C64 needs N1 == N2 == N3 <= 24              */
  double lattice[9];      /* rows a1, a2, a3 (bohr), row-major                                   */
  int nk;                 /* number of k-points (>= 1)                                           */
  const double *kpts;     /* HOST [nk][3] Cartesian k-points (bohr^-1); copied at plan creation  */
  int n_occ;              /* occupied bands per k (the j of the sum)                             */
  int n_tgt;              /* target bands per k (the i of V_x u_i)                               */
  double omega;           /* range separation (bohr^-1), > 0; the paper's mu                     */
  double alpha;           /* Fock mixing fraction, 0.25 in HSE                                   */
  double spin_degeneracy; /* g_s in E_x (2 for a closed shell); not used by V_x                  */
  int dtype;              /* HSE_C64, HSE_C128 or HSE_C64_TC                                     */
  /* Down-sampled Fock sum (Sec. II C, after Eq. "Fock-DS"): the sum over the occupied
   * orbitals' k-points k' runs over nk_occ of the nk points, kocc[0..nk_occ) (HOST, distinct
   * indices into kpts, copied at plan creation), with the weight 1/nk_occ in place of 1/nk.
   * The orbital arrays keep the full mesh; only the sampled rows of u_occ and occ are read,
   * and the VJP w.r.t. u_occ is zero at the other k-points.  nk_occ = 0: every k-point
   * (kocc ignored).  Batched plans require nk_occ = 0. */
  int nk_occ;
  const int *kocc;
} hse_problem;

typedef struct hse_plan_s *hse_plan;

/* Build a plan: validates the problem, tabulates v(|G+q|) (and d v/d omega) in FP64
 * for every distinct q = k - k' on the current device, and allocates the reduction
 * scratch.  Synchronises the device.  *out is NULL on failure. */
int hse_plan_create(hse_plan *out, const hse_problem *p);

/* Batched plan over ncells independent cells of unequal grids, k-meshes and band
 * counts (all HSE_C64, cubic grids).  hse_fock_apply_batched runs every cell's
 * pairs in one captured graph: persistent kernels over all cells' work items, or each
 * cell's single-cell launches on parallel branches, as the autotuner chooses. */
int hse_plan_create_batched(hse_plan *out, const hse_problem *cells, int ncells);

int hse_plan_destroy(hse_plan plan);

/* V_x applied to the targets (Sec. II C, Eq. "Fock-DS" with the 1/N_k weight, or 1/nk_occ
 * over the sampled k' of a down-sampled plan).
 *   u_occ  device [nk][n_occ][N]   occupied orbitals u_{j,k'}
 *   occ    device [nk][n_occ]      occupations f_{j,k'} (double)
 *   u_tgt  device [nk][n_tgt][N]   target orbitals u_{i,k}; may equal u_occ
 *   vx_out device [nk][n_tgt][N]   result, overwritten; must not overlap any input
 * Complex64 or complex128 per the plan's dtype (complex64 for HSE_C64_TC).  Complex64 pair
 * terms are summed over the bands of each k' in FP32 and over k' with compensation (TwoSum).
 * Asynchronous on `stream`, except
 * that a complex64 call running the pencil-load kernel (24^3 grids here, and the VJP with
 * respect to u_occ at every size) copies the orbitals it reads into plan scratch in a
 * pencil-blocked layout, which the first such call (or one needing more than before)
 * allocates with device-wide synchronisation. */
int hse_fock_apply(hse_plan plan, const void *u_occ, const double *occ, const void *u_tgt,
                   void *vx_out, hse_stream_t stream);

/* Fock part of E_xc (Sec. V, Eq. "Eex01"), targets = the occupied set:
 *   E_x = 1/2 g_s (1/N_k) sum_k sum_i f_{i,k} dV sum_r Re[conj(u_{i,k}) (V_x u)_{i,k}]
 * reduced in FP64 on the device.  e_x: device pointer to one double, overwritten. */
int hse_exchange_energy(hse_plan plan, const void *u_occ, const double *occ, double *e_x,
                        hse_stream_t stream);

/* Vector-Jacobian product of y = V_x[u_occ] u_tgt (PyTorch complex convention,
 * grad = dL/dRe + i dL/dIm).  With c_j = alpha f_{j,k'}/N_k, K_q = F^-1 diag(v) F,
 * phi_ji = K_q(conj(u_j) u_i), psibar_ji = K_q(conj(u_j) ybar_i):
 *   grad_u_tgt[k,i]  = -sum_{k',j} c_j u_j psibar_ji            (V_x applied to ybar)
 *   grad_u_occ[k',j] = -sum_{k,i} c_j [conj(phi_ji) ybar_i + u_i conj(psibar_ji)]
 *   grad_omega       = Re sum conj(ybar) (dV_x/domega) u_tgt
 * grad_vx is ybar.  All gradients are overwritten (not accumulated); any of the three
 * outputs may be NULL to skip it.  Outputs must not overlap inputs.  A down-sampled plan
 * writes zeros to the rows of grad_u_occ at k-points outside kocc. */
int hse_fock_apply_vjp(hse_plan plan, const void *u_occ, const double *occ, const void *u_tgt,
                       const void *grad_vx, void *grad_u_occ, void *grad_u_tgt,
                       double *grad_omega, hse_stream_t stream);

/* Batched V_x for a plan from hse_plan_create_batched: arrays of ncells HOST-side
 * pointers, each to that cell's device buffers (same layouts as hse_fock_apply).  The first
 * call autotunes the shape of the launch on the real inputs (synchronising the stream).  For
 * the persistent form: the k'-split granularity of the work items (1, 2, 4), the pencil layout
 * of the 24^3 cells (one pencil per thread or the ragged two-pencil form), the pencil layout of
 * each staged grid side (one or two pencils per thread), and whether the two persistent
 * kernels (24^3 cells; the other sides) run at once on two streams or one after the other
 * (coordinate descent from the defaults); then the per-cell form, in which every cell runs the
 * launches of a single-cell plan, on three streams forked from `stream` and joined back.  At
 * most ten timed runs.  The chosen form is captured as a CUDA graph that later calls replay.
 * The persistent form reads each call's pointers from a device table, so its graph serves
 * every call; the per-cell form passes them as launch arguments, so a call whose pointers
 * differ from those of the captured graph captures it again (host work, no synchronisation
 * beyond the first call's).  With the environment variable HSE_AUTOTUNE_CACHE naming a file,
 * the choice is stored there per GPU and cell list and read back by later plans instead of
 * timing (the first call of such a plan in the per-cell form runs once uncaptured, so that
 * its cells' scratch exists before the capture). */
int hse_fock_apply_batched(hse_plan plan, const void *const *u_occ, const double *const *occ,
                           const void *const *u_tgt, void *const *vx_out, hse_stream_t stream);

/* Kinetic term of the velocity-gauge Kohn-Sham Hamiltonian (Sec. II A, Eq. "tdks-h": the
 * (-i grad + e A(t)/c)^2 / 2m term, atomic units with e/c absorbed into A) on the periodic
 * parts:  out_{b,k}(r) = sum_G 1/2 |G + k + A|^2 u~_{b,k}(G) e^{iG.r}.  Used with V_x by the
 * Taylor propagator of Sec. II C.
 *   u, out  device [nk][nbands][N] (the plan's dtype); must not overlap
 *   A       HOST [3] vector potential (bohr^-1) */
int hse_kinetic_apply(hse_plan plan, const void *u, int nbands, const double *A, void *out,
                      hse_stream_t stream);

/* Synchronises the stream, then returns HSE_OK, HSE_ERR_TIMEOUT, HSE_ERR_SINGULAR or
 * HSE_ERR_DEVICE from the plan's device status word (and clears it), or HSE_ERR_CUDA.  Every device-side wait of
 * the library is bounded (about one second); on expiry the kernel records HSE_ERR_TIMEOUT,
 * stops waiting and returns, so the context stays usable.  Test hook: a plan created while
 * the environment variable HSE_INJECT_SKIP_FILL=1 is set never issues the first asynchronous
 * partner copy of its complex64 kernels, so that wait runs out (its results are garbage). */
int hse_status(hse_plan plan, hse_stream_t stream);

/* 1 if this build has a kernel for axis length n (and dtype), else 0. */
int hse_grid_supported(int n, int dtype);

/* Number of kernels this library has launched since load (for launch accounting). */
uint64_t hse_kernel_launches(void);

const char *hse_strerror(int code);

/* Exchange energy for callers that cannot allocate device memory: no counterpart in the
 * paper; it computes the same E_x as hse_exchange_energy (HSE_C64, cubic grids) without a
 * plan and without any allocation.
 *
 * Who needs it: an application whose device memory belongs to another allocator (a
 * framework's memory pool, a fixed per-process budget) that it may not grow, or a
 * latency-critical loop where cudaMalloc/cudaFree would synchronise the device.  Plans
 * allocate, so those callers cannot use hse_plan_create.
 *
 * Scratch: one static __device__ array of HSE_NOALLOC_SCRATCH_BYTES (4 MiB) that every GPU
 * loading this library holds until the process exits.  It must hold
 *   256 + align256(4 nk^2) + align256(4 nk^2 N) + align256(8 nk n_occ) bytes
 * (N = grid points, align256 rounds up to 256), and nk must be at most 128; larger problems
 * return HSE_ERR_INVALID_ARG before any device work.  Example: a 12^3 grid with 8 k-points
 * needs about 0.44 MiB, a 24^3 grid with 8 k-points about 3.4 MiB.
 * Set-up: the first call on each device (and the first after that device's context has been
 * replaced, e.g. by cudaDeviceReset) looks up the array's device address with
 * cudaGetSymbolAddress, with that device current; make that first call before any stream
 * capture.  All calls share the one array and each call clears or overwrites all of it that
 * it reads, but calls that overlap on the GPU (other streams, other host threads) race on it:
 * serialise them.  p->kpts is read on the host during the call and reaches the kernels by
 * value (the call copies nothing from host memory); u_occ, occ and e_x are device pointers
 * as for hse_exchange_energy.  Asynchronous on `stream`.  There is no plan, so no status
 * word for hse_status: if a bounded device-side wait of the call gives up, *e_x is set to NaN
 * (the test hook HSE_INJECT_SKIP_FILL=1 of hse_status applies here too, read at each call). */
#define HSE_NOALLOC_SCRATCH_BYTES (4u << 20)
int hse_exchange_energy_noalloc(const hse_problem *p, const void *u_occ, const double *occ,
                                double *e_x, hse_stream_t stream);

/* One fourth-order Taylor step of the time-dependent Kohn-Sham equation (Sec. II C, "time
 * evolution": the propagator exp[h dt / i] expanded to fourth order, with the Hamiltonian at
 * t + dt/2 taken at t, the choice the paper reports as sufficient for HSE):
 *   psi_out = sum_{n=0}^{4} (-i dt h)^n / n! psi,   h = T[A] + v_loc + V_x[psi]
 * with T the velocity-gauge kinetic term of hse_kinetic_apply, v_loc a real local potential
 * (e.g. the Hartree potential of hse_hartree_potential for psi) and V_x built from psi itself
 * (the plan's occupied set) with occupations occ; the Hamiltonian is frozen over the step.
 *   psi, psi_out device [nk][n_occ][N] (the plan's dtype; the plan must have n_tgt == n_occ);
 *                must not overlap
 *   occ          device [nk][n_occ]
 *   A            HOST [3] vector potential at the start of the step (bohr^-1)
 *   vloc         device double [N] local potential on the grid, or NULL for none
 * The first call allocates three orbital-sized scratch arrays in the plan (device-wide
 * synchronisation); later calls are asynchronous on `stream`.  Not for batched plans. */
int hse_taylor_step(hse_plan plan, const void *psi, const double *occ, const double *A, double dt,
                    const double *vloc, void *psi_out, hse_stream_t stream);

/* Hartree potential of the orbitals' density (Sec. II A, Eq. "tdks-h"; Poisson's equation in
 * atomic units with a neutralising background):
 *   rho(r) = sum_{k,i} (g_s f_{i,k} / N_k) |u_{i,k}(r)|^2,
 *   v_H(r) = sum_{G != 0} 4 pi rho~(G) / |G|^2 e^{iG.r},  rho~ = (1/N) sum_r rho e^{-iG.r},
 * in FP64 (density, transforms and scaling).  The Hartree energy of Eq. "Eex01" is
 * 1/2 dV sum_r v_H rho.
 *   psi  device [nk][n_occ][N] (the plan's dtype), occ device [nk][n_occ]
 *   vh   device double [N], overwritten
 * g_s is the plan's spin_degeneracy.  The first call allocates an N-point FP64 work array in
 * the plan; later calls are asynchronous on `stream`.  Not for batched plans. */
int hse_hartree_potential(hse_plan plan, const void *psi, const double *occ, double *vh,
                          hse_stream_t stream);

/* Spatially averaged electric current of the orbitals (Sec. II A, Eqs. "current_dns" and
 * "current_elec", without J_NL, the nonlocal pseudopotential part; atomic units, e/c
 * absorbed into A):
 *   J = -(1/Omega) int_Omega sum_i w_i Re[psi_i* (-i grad + A) psi_i]
 *     = -sum_{k,i} (g_s f_{i,k} / N_k) sum_G |c_{i,k}(G)|^2 (G + k + A),
 * c = (1/N) sum_r u(r) e^{-iG.r}, computed with FP64 transforms and reduced in FP64.
 *   psi  device [nk][n_occ][N] (the plan's dtype), occ device [nk][n_occ]
 *   A    HOST [3];  J  device double[3], overwritten
 * g_s is the plan's spin_degeneracy.  The first call allocates an FP64 copy of the orbitals
 * in the plan; later calls are asynchronous on `stream`.  Not for batched plans. */
int hse_current(hse_plan plan, const void *psi, const double *occ, const double *A, double *J,
                hse_stream_t stream);

/* Overlap matrices of a set of orbitals, in FP64 (products and sums; complex64 orbitals are
 * widened on load).  With cell normalisation, as everywhere in this interface:
 *   S[k][a][b] = dV sum_r conj(u_{a,k}(r)) u_{b,k}(r),   dV = Omega / N.
 * The 4th-order Taylor step (Sec. II C) is not unitary: max |S - 1| of the propagated
 * orbitals is the check of a propagation.
 *   u  device [nk][nbands][N] (the plan's dtype), nbands >= 1
 *   S  device double [nk][nbands][nbands][2] (real, imaginary), overwritten; S[k][b][a] is
 *      the conjugate of S[k][a][b] and the diagonal is real
 * Asynchronous on `stream`.  Not for batched plans. */
int hse_overlap(hse_plan plan, const void *u, int nbands, double *S, hse_stream_t stream);

/* Orthonormalises the bands of every k-point in place, in band order: modified Gram-Schmidt
 * (band a loses its component along each earlier band b < a in turn, then is divided by its
 * norm), applied twice, with every inner product and update in FP64.  complex64 orbitals are
 * widened into an FP64 copy and rounded once when written back; complex128 ones are updated
 * in place.  A band that is linearly dependent on the earlier ones (its norm after the
 * projections at most 1e-12 of its norm before them for complex128, 1e-5 for complex64, whose
 * rounding leaves about 1e-7 of any band outside the span of the others) is set to zero and
 * the plan's status word records HSE_ERR_SINGULAR (returned by hse_status).
 *   u  device [nk][nbands][N] (the plan's dtype), 1 <= nbands <= 4096, overwritten
 * complex64: the first call (or one with more bands than before) allocates an FP64 copy of
 * the orbitals in the plan (device-wide synchronisation).  Asynchronous on `stream`
 * otherwise.  Not for batched plans. */
int hse_orthonormalize(hse_plan plan, void *u, int nbands, hse_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* HSE_FOCK_H */
