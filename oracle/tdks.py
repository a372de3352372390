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


def hamiltonian_apply(psi_frozen, occ, phi, kpts, lattice, grid, A, omega, alpha) -> np.ndarray:
    """h phi = T[A] phi + V_x[psi_frozen] phi."""
    return kinetic_apply(phi, kpts, lattice, grid, A) + ho.fock_apply(
        psi_frozen, occ, phi, kpts, lattice, grid, omega, alpha)


def taylor_step(psi, occ, kpts, lattice, grid, A, omega, alpha, dt, order: int = 4) -> np.ndarray:
    """sum_{n=0}^{order} (-i dt h)^n / n! psi with h frozen at psi (Sec. II C)."""
    out = np.array(psi, dtype=np.complex128, copy=True)
    term = out.copy()
    for n in range(1, order + 1):
        term = (-1j * dt / n) * hamiltonian_apply(psi, occ, term, kpts, lattice, grid, A, omega, alpha)
        out = out + term
    return out


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
