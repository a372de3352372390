"""FP64 CPU oracle of the Taylor-series time step of the TDKS equation (test infrastructure).

Only ``tests/`` may use it.  Follows arXiv:1507.05156:

* Sec. II A, Eq. "tdks-h": velocity-gauge kinetic term (-i grad + e A(t)/c)^2 / 2m; in atomic
  units with e/c absorbed into A it acts on the periodic part u_{b,k} as
      (T u)(r) = sum_G 1/2 |G + k + A|^2 u~(G) e^{iG.r};
  A(t) = -c int^t E(t') dt', i.e. A(t) = -E t for a field E switched on at t = 0.
* Sec. II C (time evolution): psi(t + dt) = sum_{n=0}^{4} (h dt / i)^n / n! psi(t), with the
  Hamiltonian at t + dt/2 approximated by the one at t (the choice the paper reports as
  sufficient for HSE).  The synthetic Hamiltonian used here is h = T[A(t)] + V_x[psi(t)]:
  the pseudopotential, Hartree and semilocal terms of the paper need data that is not here.
* Sec. II A, Eqs. "current_dns" / "current_elec": the spatially averaged electric current
  J(t) = -(1/Omega) int_Omega j dr, j = sum_i Re[psi_i* (-i grad + A) psi_i] (atomic units,
  e = m = hbar = 1, e/c absorbed), without the pseudopotential's nonlocal part J_NL.  Each
  orbital counts with g_s f_{i,k} / N_k.  With psi = e^{ik.r} u, u = sum_G c_G e^{iG.r}
  (c = the 1/N forward transform), int_Omega psi* (-i grad + A) psi = Omega sum_G |c_G|^2
  (G + k + A), so J = -sum_{k,i} (g_s f_{i,k} / N_k) sum_G |c_G|^2 (G + k + A).
* Sec. II A (Eq. "tdks-h") and Sec. V (Eq. "Eex01"): the Hartree potential v_H of the density
  rho(r) = sum_{k,i} (g_s f_{i,k} / N_k) |u_{i,k}(r)|^2, from Poisson's equation in atomic
  units, -lap v_H = 4 pi (rho - rho_avg): v_H(G) = 4 pi rho~(G) / |G|^2, v_H(G = 0) = 0 (the
  neutralising background), and the Hartree energy per cell 1/2 int_Omega v_H rho.  A local
  potential v_loc(r) (v_H here) enters h as a multiplication.
* Sec. IV (laser pulse): A(t) = -(E0 / w) cos(w t) sin^2(pi t / T_d) along a direction for
  0 < t < T_d (zero otherwise), E(t) = -dA/dt, and the energy given to the electrons per unit
  volume W(t) = int^t J(t') . E(t') dt' (Eq. for W in Sec. V).
"""
from __future__ import annotations

import math

import numpy as np

from . import hse_oracle as ho


def kinetic_apply(u, kpts, lattice, grid, A) -> np.ndarray:
    """1/2 |G + k + A|^2 applied to u [nk][nb][grid] (Fourier-diagonal)."""
    grid = tuple(int(g) for g in grid)
    u = np.asarray(u, dtype=np.complex128).reshape(np.shape(u)[:2] + grid)
    G = ho.g_vectors(grid, lattice)
    out = np.empty_like(u)
    for k in range(u.shape[0]):
        gk = G + np.asarray(kpts[k]) + np.asarray(A, dtype=np.float64)
        fac = 0.5 * np.sum(gk * gk, axis=-1)
        out[k] = ho.inverse_transform(ho.forward_transform(u[k]) * fac)
    return out


def hamiltonian_apply(psi_frozen, occ, phi, kpts, lattice, grid, A, omega, alpha, vloc=None) -> np.ndarray:
    """h phi = T[A] phi + v_loc phi + V_x[psi_frozen] phi (v_loc: a real grid, or None)."""
    out = kinetic_apply(phi, kpts, lattice, grid, A) + ho.fock_apply(
        psi_frozen, occ, phi, kpts, lattice, grid, omega, alpha)
    if vloc is not None:
        grid = tuple(int(g) for g in grid)
        out = out + np.asarray(vloc, dtype=np.float64).reshape(grid) * np.asarray(phi).reshape(out.shape)
    return out


def taylor_step(psi, occ, kpts, lattice, grid, A, omega, alpha, dt, order: int = 4, vloc=None) -> np.ndarray:
    """sum_{n=0}^{order} (-i dt h)^n / n! psi with h frozen at psi (Sec. II C)."""
    out = np.array(psi, dtype=np.complex128, copy=True)
    term = out.copy()
    for n in range(1, order + 1):
        term = (-1j * dt / n) * hamiltonian_apply(psi, occ, term, kpts, lattice, grid, A, omega, alpha, vloc)
        out = out + term
    return out


def density(u, occ, grid, spin_degeneracy: float = 2.0) -> np.ndarray:
    """rho(r) = sum_{k,i} (g_s f_{i,k} / N_k) |u_{i,k}(r)|^2 (electrons per bohr^3)."""
    grid = tuple(int(g) for g in grid)
    u = np.asarray(u, dtype=np.complex128).reshape(np.shape(u)[:2] + grid)
    occ = np.asarray(occ, dtype=np.float64)
    return spin_degeneracy / u.shape[0] * np.einsum("kb,kbxyz->xyz", occ, np.abs(u) ** 2)


def hartree_potential(u, occ, lattice, grid, spin_degeneracy: float = 2.0) -> np.ndarray:
    """v_H(r) = sum_{G != 0} 4 pi rho~(G) / |G|^2 e^{iG.r}, real [N1][N2][N3]."""
    grid = tuple(int(g) for g in grid)
    rho_t = ho.forward_transform(density(u, occ, grid, spin_degeneracy))
    G = ho.g_vectors(grid, lattice)
    g2 = np.sum(G * G, axis=-1)
    fac = np.zeros_like(g2)
    nz = g2 > 0
    fac[nz] = 4.0 * np.pi / g2[nz]
    return np.real(ho.inverse_transform(rho_t * fac))


def hartree_energy(u, occ, lattice, grid, spin_degeneracy: float = 2.0) -> float:
    """E_H = 1/2 int_Omega v_H rho dr per cell (Eq. Eex01), by the grid sum with dV = Omega / N."""
    grid = tuple(int(g) for g in grid)
    rho = density(u, occ, grid, spin_degeneracy)
    vh = hartree_potential(u, occ, lattice, grid, spin_degeneracy)
    dV = ho.cell_volume(lattice) / np.prod(grid)
    return float(0.5 * dV * np.sum(vh * rho))


def propagate(psi0, occ, kpts, lattice, grid, omega, alpha, dt, nsteps, efield) -> np.ndarray:
    """nsteps Taylor steps; step s uses A(t_s) = -efield * t_s, t_s = s dt."""
    psi = np.array(psi0, dtype=np.complex128, copy=True)
    E = np.asarray(efield, dtype=np.float64)
    for s in range(nsteps):
        psi = taylor_step(psi, occ, kpts, lattice, grid, -E * (s * dt), omega, alpha, dt)
    return psi


def taylor_norm_factor(x: float, order: int = 4) -> float:
    """|sum_{n<=order} (-i x)^n / n!|^2 for real x (the truncated series on an eigenvector)."""
    s = sum((-1j * x) ** n / math.factorial(n) for n in range(order + 1))
    return float(abs(s) ** 2)


def current(u, occ, kpts, lattice, grid, A, spin_degeneracy: float = 2.0) -> np.ndarray:
    """J = -sum_{k,i} (g_s f_{i,k} / N_k) sum_G |c_G|^2 (G + k + A), c = forward transform of
    u_{i,k} (Eqs. current_dns / current_elec without J_NL), a 3-vector."""
    grid = tuple(int(g) for g in grid)
    u = np.asarray(u, dtype=np.complex128).reshape(np.shape(u)[:2] + grid)
    occ = np.asarray(occ, dtype=np.float64)
    G = ho.g_vectors(grid, lattice)
    nk = u.shape[0]
    J = np.zeros(3)
    for k in range(nk):
        gk = G + np.asarray(kpts[k]) + np.asarray(A, dtype=np.float64)       # [grid][3]
        c = ho.forward_transform(u[k])                                        # [nb][grid]
        w = np.abs(c) ** 2
        J -= spin_degeneracy / nk * np.einsum("b,bxyz,xyzc->c", occ[k], w, gk)
    return J


def pulse_vector_potential(t: float, E0: float, w: float, Td: float, direction) -> np.ndarray:
    """A(t) = -(E0 / w) cos(w t) sin^2(pi t / T_d) d for 0 <= t <= T_d, else 0 (Sec. IV)."""
    d = np.asarray(direction, dtype=np.float64)
    if t <= 0.0 or t >= Td:
        return np.zeros(3)
    return -(E0 / w) * math.cos(w * t) * math.sin(math.pi * t / Td) ** 2 * d


def pulse_field(t: float, E0: float, w: float, Td: float, direction) -> np.ndarray:
    """E(t) = -dA/dt of pulse_vector_potential, differentiated by hand."""
    d = np.asarray(direction, dtype=np.float64)
    if t <= 0.0 or t >= Td:
        return np.zeros(3)
    s, c = math.sin(math.pi * t / Td), math.cos(math.pi * t / Td)
    dA = (E0 / w) * (w * math.sin(w * t) * s * s - math.cos(w * t) * 2.0 * s * c * math.pi / Td)
    return -dA * d


def propagate_pulse(psi0, occ, kpts, lattice, grid, omega, alpha, dt, nsteps, E0, w, Td, direction,
                    spin_degeneracy: float = 2.0, hartree: bool = False):
    """nsteps Taylor steps under the pulse; step s (t_s = s dt -> t_s + dt) uses h frozen at
    psi(t_s) with A(t_s) (and, with ``hartree``, v_H of psi(t_s) as a local potential).  Returns (psi, J [nsteps+1][3], W [nsteps+1]) with J_s = J(t_s)
    from psi(t_s) and A(t_s), and W by the trapezoidal rule on J . E."""
    psi = np.array(psi0, dtype=np.complex128, copy=True)
    Js, Ws = [], [0.0]
    for s in range(nsteps + 1):
        t = s * dt
        A = pulse_vector_potential(t, E0, w, Td, direction)
        Js.append(current(psi, occ, kpts, lattice, grid, A, spin_degeneracy))
        if s > 0:
            e0 = pulse_field(t - dt, E0, w, Td, direction)
            e1 = pulse_field(t, E0, w, Td, direction)
            Ws.append(Ws[-1] + 0.5 * dt * (Js[-2] @ e0 + Js[-1] @ e1))
        if s < nsteps:
            vloc = hartree_potential(psi, occ, lattice, grid, spin_degeneracy) if hartree else None
            psi = taylor_step(psi, occ, kpts, lattice, grid, A, omega, alpha, dt, vloc=vloc)
    return psi, np.array(Js), np.array(Ws)
