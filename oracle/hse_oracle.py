"""FP64 CPU oracle of the HSE short-range Fock-like exchange operator.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import or call this
module; it is used by ``tests/``, by ``__graft_entry__.smoke()`` and by the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  It shares no code with
the CUDA library: its only inputs are arrays from the seeded generators.

It is written to be read against the paper (Sato, Taniguchi, Shinohara, Yabana,
arXiv:1507.05156, Sec. II C "Nonlocal Fock-like term"), not to be fast:

* real-space definition (Sec. II C, first equation of the subsection):
      v^{SR,Fock} psi_i(r) = sum_{j occ} int dr' v_SR(r - r') psi_j(r) psi_j*(r') psi_i(r');
* Fourier-space form (Eq. "Fock"):
      v^{SR,Fock} psi_i(r) = sum_{j occ} psi_j(r) [F^-1 v~^SR(G) rho~_ji(G)](r),
      rho_ji = psi_j* psi_i;
* k/band decomposition (Eq. "Fock-DS"): i -> (k, b), j -> (k', b').

Readings (where the paper is silent, garbled or at odds with itself):

1. Short-range kernel: the text names erf(mu r)/r but calls it short-ranged; the
   short-range part of HSE is erfc(omega r)/r, whose transform is
   v~(g) = 4 pi / g^2 (1 - exp(-g^2 / 4 omega^2)), finite at g = 0 (pi / omega^2).
2. Sign and mixing: exchange enters with -alpha (alpha = 1/4 in HSE, Sec. II B).
3. Discrete Fourier convention on the N1 x N2 x N3 grid: forward
   rho~(G_m) = (1/N) sum_r rho(r) e^{-i G_m . r}, inverse sum_m (.) e^{+i G_m . r}
   with no factor; G_m = m1 b1 + m2 b2 + m3 b3, m_d in numpy fftfreq order
   (so the Nyquist index of an even axis is m = -N_d/2).
4. Bloch form: u_{b,k} are the periodic parts, cell-normalised dV sum |u|^2 = 1.
   With q = k - k' (not folded to the first zone) the periodic part of the result is
      (V_x u)_{i,k}(r) = -alpha (1/N_k) sum_{k'} sum_j f_{j,k'} u_{j,k'}(r)
                          sum_m v~(|G_m + q|) rho~_ji(G_m) e^{i G_m . r},
      rho_ji(r) = conj(u_{j,k'}(r)) u_{i,k}(r).
   The uniform k-weight 1/N_k is the one the down-sampling equation leaves out.
5. Occupations f in [0,1] per spin-orbital; the spin degeneracy g_s enters E_x only.
6. Exchange energy (the Fock part of E_xc in Eq. "Eex01"):
      E_x = 1/2 g_s (1/N_k) sum_k sum_{i occ} f_{i,k} dV sum_r Re[conj(u_{i,k}) (V_x u)_{i,k}],
   with the targets equal to the occupied set.
7. Down-sampling (Sec. II C, after Eq. "Fock-DS"): the sum over the occupied orbitals'
   k-points k' runs over a sub-mesh of N_q of the N_k points of the orbital mesh, with the
   uniform weight 1/N_q in place of 1/N_k ("kocc" below: the indices of the sampled points;
   None = all).  The targets keep the full mesh.

Every function below works in float64 / complex128.
"""
from __future__ import annotations

import os
from typing import Optional, Sequence, Tuple

import numpy as np
import scipy.fft as sfft


def _workers() -> int:
    return int(os.environ.get("HSE_ORACLE_WORKERS", os.cpu_count() or 1))


# ---------------------------------------------------------------------------
# Geometry (reading 3)
# ---------------------------------------------------------------------------

def reciprocal_rows(lattice: np.ndarray) -> np.ndarray:
    """Rows b1, b2, b3 with a_i . b_j = 2 pi delta_ij."""
    A = np.asarray(lattice, dtype=np.float64)
    return 2.0 * np.pi * np.linalg.inv(A).T


def cell_volume(lattice: np.ndarray) -> float:
    return float(abs(np.linalg.det(np.asarray(lattice, dtype=np.float64))))


def integer_frequencies(n: int) -> np.ndarray:
    """m_d of array index 0..n-1: 0, 1, ..., ceil(n/2)-1, -floor(n/2), ..., -1."""
    idx = np.arange(n)
    return np.where(idx <= (n - 1) // 2, idx, idx - n)


def g_vectors(grid: Sequence[int], lattice: np.ndarray) -> np.ndarray:
    """Cartesian G_m for every grid index in FFT order, shape [N1][N2][N3][3]."""
    b = reciprocal_rows(lattice)
    m1, m2, m3 = np.meshgrid(*(integer_frequencies(int(n)) for n in grid), indexing="ij")
    return m1[..., None] * b[0] + m2[..., None] * b[1] + m3[..., None] * b[2]


# ---------------------------------------------------------------------------
# The short-range screened Coulomb kernel (reading 1)
# ---------------------------------------------------------------------------

def screened_kernel(g2: np.ndarray, omega: float) -> np.ndarray:
    """v~(g) = 4 pi / g^2 (1 - exp(-g^2 / (4 omega^2))), v~(0) = pi / omega^2.

    Written as (pi / omega^2) * (-expm1(-x) / x), x = g^2 / (4 omega^2), which has no
    cancellation for small g.
    """
    g2 = np.asarray(g2, dtype=np.float64)
    x = g2 / (4.0 * omega * omega)
    out = np.empty_like(x)
    small = x == 0.0
    out[small] = 1.0
    xs = x[~small]
    out[~small] = -np.expm1(-xs) / xs
    return (np.pi / (omega * omega)) * out


def screened_kernel_domega(g2: np.ndarray, omega: float) -> np.ndarray:
    """d v~ / d omega = -(2 pi / omega^3) exp(-g^2 / (4 omega^2))."""
    g2 = np.asarray(g2, dtype=np.float64)
    return -(2.0 * np.pi / omega ** 3) * np.exp(-g2 / (4.0 * omega * omega))


def kernel_on_grid(grid, lattice, q, omega, derivative: bool = False) -> np.ndarray:
    """v~(|G_m + q|) (or its omega derivative) on the FFT-ordered grid."""
    G = g_vectors(grid, lattice) + np.asarray(q, dtype=np.float64)
    g2 = np.sum(G * G, axis=-1)
    return screened_kernel_domega(g2, omega) if derivative else screened_kernel(g2, omega)


# ---------------------------------------------------------------------------
# The pipeline steps of Eq. "Fock", in the paper's order
# ---------------------------------------------------------------------------

def pair_density(u_j: np.ndarray, u_i: np.ndarray) -> np.ndarray:
    """rho_ji(r) = psi_j*(r) psi_i(r) (Bloch phase carried by q, reading 4)."""
    return np.conj(u_j) * u_i


def forward_transform(rho: np.ndarray) -> np.ndarray:
    """rho~(G_m) = (1/N) sum_r rho(r) e^{-i G_m . r} over the last three axes."""
    return sfft.fftn(rho, axes=(-3, -2, -1), norm="forward", workers=_workers())


def inverse_transform(rt: np.ndarray) -> np.ndarray:
    """phi(r) = sum_m rt(G_m) e^{+i G_m . r} over the last three axes."""
    return sfft.ifftn(rt, axes=(-3, -2, -1), norm="forward", workers=_workers())


def _as_grid(u: np.ndarray, grid) -> np.ndarray:
    u = np.asarray(u)
    return u.reshape(u.shape[:2] + tuple(int(g) for g in grid)).astype(np.complex128, copy=False)


def _sampled(kocc, nk):
    """k' indices of the Fock sum (reading 7): all nk points, or the sampled sub-mesh."""
    if kocc is None:
        return list(range(nk))
    kocc = [int(k) for k in kocc]
    if not kocc or len(set(kocc)) != len(kocc) or min(kocc) < 0 or max(kocc) >= nk:
        raise ValueError("kocc must list distinct k-point indices")
    return kocc


def fock_apply(u_occ, occ, u_tgt, kpts, lattice, grid, omega, alpha,
               targets: Optional[Sequence[Tuple[int, int]]] = None,
               kernel: str = "value", kocc: Optional[Sequence[int]] = None) -> np.ndarray:
    """(V_x u)_{i,k} for every target, reading 4 (reading 7 when ``kocc`` is given).

    u_occ [nk][n_occ][N1][N2][N3], occ [nk][n_occ], u_tgt [nk][n_tgt][...],
    kpts [nk][3] Cartesian.  ``targets`` optionally restricts the output to a list
    of (k, i); the result is then [len(targets)][N1][N2][N3], otherwise it is
    [nk][n_tgt][N1][N2][N3].  ``kernel='domega'``
    replaces v~ by d v~/d omega (the omega derivative of the operator).  ``kocc`` lists the
    k-points whose occupied orbitals enter the sum (weight 1 / len(kocc)).
    """
    grid = tuple(int(g) for g in grid)
    u_occ = _as_grid(u_occ, grid)
    u_tgt = _as_grid(u_tgt, grid)
    occ = np.asarray(occ, dtype=np.float64)
    kpts = np.asarray(kpts, dtype=np.float64)
    nk = kpts.shape[0]
    kps = _sampled(kocc, nk)
    full = targets is None
    if full:
        targets = [(k, i) for k in range(nk) for i in range(u_tgt.shape[1])]
    out = np.zeros((len(targets),) + grid, dtype=np.complex128)
    by_k = {}
    for t, (k, i) in enumerate(targets):
        by_k.setdefault(k, []).append((t, i))
    for k, items in by_k.items():
        rows = [t for t, _ in items]
        u_i = u_tgt[k, [i for _, i in items]]                  # [T][grid]
        acc = np.zeros_like(u_i)
        for kp in kps:
            q = kpts[k] - kpts[kp]
            v = kernel_on_grid(grid, lattice, q, omega, derivative=(kernel == "domega"))
            u_j = u_occ[kp]                                    # [J][grid]
            rho = pair_density(u_j[:, None], u_i[None, :])     # [J][T][grid]
            rt = forward_transform(rho) * v
            phi = inverse_transform(rt)
            acc += np.einsum("j,j...,jt...->t...", occ[kp], u_j, phi)
        out[rows] = -alpha / len(kps) * acc
    if full:
        return out.reshape(u_tgt.shape)
    return out


def exchange_energy(u_occ, occ, kpts, lattice, grid, omega, alpha, spin_degeneracy=2.0,
                    kocc: Optional[Sequence[int]] = None) -> float:
    """E_x of reading 6, with the targets equal to the occupied orbitals (all N_k points);
    ``kocc`` down-samples the Fock sum inside V_x (reading 7)."""
    grid = tuple(int(g) for g in grid)
    u_occ = _as_grid(u_occ, grid)
    nk, n_occ = u_occ.shape[:2]
    vx = fock_apply(u_occ, occ, u_occ, kpts, lattice, grid, omega, alpha, kocc=kocc)
    dV = cell_volume(lattice) / np.prod(grid)
    e = 0.0
    for k in range(nk):
        for i in range(n_occ):
            e += occ[k][i] * dV * np.real(np.vdot(u_occ[k, i], vx[k, i]))
    return 0.5 * spin_degeneracy * e / nk


def fock_apply_vjp(u_occ, occ, u_tgt, grad_vx, kpts, lattice, grid, omega, alpha,
                   kocc: Optional[Sequence[int]] = None):
    """Vector-Jacobian product of y = V_x[u_occ] u_tgt (PyTorch complex convention).

    With ybar = grad_vx, c_j = alpha f_{j,k'} / N_k, K_q = F^-1 diag(v~(|G+q|)) F,
    phi_ji = K_q(conj(u_j) u_i) and psibar_ji = K_q(conj(u_j) ybar_i):

      d/d u_tgt[k,i]  = -sum_{k',j} c_j u_j psibar_ji            ( = V_x applied to ybar )
      d/d u_occ[k',j] = -sum_{k,i}  c_j [conj(phi_ji) ybar_i + u_i conj(psibar_ji)]
      d/d omega       = Re sum_{k,i} sum_r conj(ybar_i) (-sum_{k',j} c_j u_j K'_q(rho_ji)),
                        K'_q with v~ replaced by d v~ / d omega.

    For a real-linear map dy = A dz + B conj(dz) the gradient is A^H ybar + B^T conj(ybar);
    K_q is Hermitian because v~ is real.  With ``kocc`` (reading 7) k' runs over the sampled
    points, N_k becomes N_q in c_j, and the rows of g_occ at k-points outside the sub-mesh
    are zero.  Returns (g_occ, g_tgt, g_omega).
    """
    grid = tuple(int(g) for g in grid)
    u_occ = _as_grid(u_occ, grid)
    u_tgt = _as_grid(u_tgt, grid)
    ybar = _as_grid(grad_vx, grid)
    occ = np.asarray(occ, dtype=np.float64)
    kpts = np.asarray(kpts, dtype=np.float64)
    nk = kpts.shape[0]
    kps = _sampled(kocc, nk)
    g_occ = np.zeros_like(u_occ)
    g_tgt = np.zeros_like(u_tgt)
    g_omega = 0.0
    for k in range(nk):
        u_i = u_tgt[k]
        y_i = ybar[k]
        for kp in kps:
            q = kpts[k] - kpts[kp]
            v = kernel_on_grid(grid, lattice, q, omega)
            dv = kernel_on_grid(grid, lattice, q, omega, derivative=True)
            u_j = u_occ[kp]
            c = alpha * occ[kp] / len(kps)                           # [J]
            rho_t = forward_transform(pair_density(u_j[:, None], u_i[None, :]))
            sig_t = forward_transform(pair_density(u_j[:, None], y_i[None, :]))
            phi = inverse_transform(rho_t * v)                        # [J][T][grid]
            psib = inverse_transform(sig_t * v)
            dphi = inverse_transform(rho_t * dv)
            g_tgt[k] += -np.einsum("j,j...,jt...->t...", c, u_j, psib)
            g_occ[kp] += -np.einsum("j,jt...->j...", c,
                                    np.conj(phi) * y_i[None, :] + u_i[None, :] * np.conj(psib))
            dy = -np.einsum("j,j...,jt...->t...", c, u_j, dphi)
            g_omega += float(np.real(np.vdot(y_i, dy)))
    return g_occ, g_tgt, g_omega


# ---------------------------------------------------------------------------
# Brute-force real-space form (first equation of Sec. II C), tiny grids only
# ---------------------------------------------------------------------------

def periodic_kernel_realspace(grid, lattice, q, omega) -> np.ndarray:
    """K_q(d) = sum_m v~(|G_m + q|) e^{i G_m . r_d} for every grid offset d, by explicit
    summation over m (no FFT): the band-limited periodic image of v_SR on the grid."""
    grid = tuple(int(g) for g in grid)
    v = kernel_on_grid(grid, lattice, q, omega).reshape(-1)
    ms = np.stack(np.meshgrid(*(integer_frequencies(n) for n in grid), indexing="ij"), -1).reshape(-1, 3)
    ds = np.stack(np.meshgrid(*(np.arange(n) for n in grid), indexing="ij"), -1).reshape(-1, 3)
    phase = 2.0 * np.pi * (ds[:, None, :] / np.array(grid)) * ms[None, :, :]
    return (np.exp(1j * phase.sum(-1)) @ v).reshape(grid)


def fock_apply_realspace(u_occ, occ, u_tgt, kpts, lattice, grid, omega, alpha,
                         kocc: Optional[Sequence[int]] = None) -> np.ndarray:
    """O(N^2) double sum  -alpha/N_k sum_{k',j} f u_j(r) (1/N) sum_{r'} K_q(r-r') rho_ji(r')
    (N_k -> N_q and k' over the sub-mesh with ``kocc``, reading 7)."""
    grid = tuple(int(g) for g in grid)
    u_occ = _as_grid(u_occ, grid)
    u_tgt = _as_grid(u_tgt, grid)
    nk, n_tgt = u_tgt.shape[:2]
    N = int(np.prod(grid))
    idx = np.stack(np.meshgrid(*(np.arange(n) for n in grid), indexing="ij"), -1).reshape(-1, 3)
    diff = (idx[:, None, :] - idx[None, :, :]) % np.array(grid)       # [N][N][3]
    kps = _sampled(kocc, nk)
    out = np.zeros((nk, n_tgt, N), dtype=np.complex128)
    for k in range(nk):
        for kp in kps:
            K = periodic_kernel_realspace(grid, lattice, kpts[k] - kpts[kp], omega)
            M = K[diff[..., 0], diff[..., 1], diff[..., 2]] / N          # [N][N]
            for i in range(n_tgt):
                ui = u_tgt[k, i].reshape(-1)
                for j in range(u_occ.shape[1]):
                    uj = u_occ[kp, j].reshape(-1)
                    out[k, i] += -alpha / len(kps) * occ[kp][j] * uj * (M @ (np.conj(uj) * ui))
    return out.reshape((nk, n_tgt) + grid)


def direct_dft(x: np.ndarray) -> np.ndarray:
    """(1/N) sum_r x(r) e^{-i G_m . r} by an explicit O(N^2) sum over a 3-D grid."""
    grid = x.shape[-3:]
    N = int(np.prod(grid))
    idx = np.stack(np.meshgrid(*(np.arange(n) for n in grid), indexing="ij"), -1).reshape(-1, 3)
    ph = np.exp(-2j * np.pi * ((idx[:, None, :] * idx[None, :, :]) / np.array(grid)).sum(-1))
    return (ph @ x.reshape(-1)).reshape(grid) / N
