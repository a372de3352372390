"""Pins of the Taylor-step oracle (Sec. II A kinetic term, Sec. II C time evolution)."""
import numpy as np
import scipy.linalg

import oracle.tdks as td
from oracle import hse_oracle as ho
from paper_1507_05156_gb300 import inputs

TRICLINIC = np.array([[7.1, 0.3, -0.4], [0.9, 6.2, 0.5], [-0.6, 1.1, 5.3]])


def _positions(grid, A):
    i1, i2, i3 = np.meshgrid(*(np.arange(n) for n in grid), indexing="ij")
    return (i1[..., None] / grid[0]) * A[0] + (i2[..., None] / grid[1]) * A[1] + (i3[..., None] / grid[2]) * A[2]


def test_kinetic_on_plane_wave_closed_form():
    grid = (6, 5, 4)
    b = 2 * np.pi * np.linalg.inv(TRICLINIC).T
    G = 2 * b[0] - 1 * b[1] + 1 * b[2]
    u = np.exp(1j * (_positions(grid, TRICLINIC) @ G))[None, None]
    k = np.array([[0.1, -0.2, 0.05]])
    A = np.array([0.03, 0.0, -0.02])
    out = td.kinetic_apply(u, k, TRICLINIC, grid, A)
    g = G + k[0] + A
    np.testing.assert_allclose(out, 0.5 * (g @ g) * u, atol=1e-12)


def test_taylor_norm_drift_closed_form():
    """alpha = 0, A = 0, a plane-wave orbital with kinetic energy e: one step multiplies it by
    sum_{n<=4} (-i e dt)^n/n!, whose squared modulus is 1 - (e dt)^6/72 + (e dt)^8/576."""
    grid = (4, 4, 4)
    A_ = inputs.cubic_lattice(6.0)
    b = 2 * np.pi / 6.0
    G = np.array([b, 0.0, -b])
    u = np.exp(1j * (_positions(grid, A_) @ G))[None, None] / np.sqrt(6.0 ** 3)
    k = np.zeros((1, 3))
    dt = 0.3
    out = td.taylor_step(u, np.ones((1, 1)), k, A_, grid, np.zeros(3), 0.2, 0.0, dt)
    e = 0.5 * G @ G
    x = e * dt
    ratio = np.vdot(out, out).real / np.vdot(u, u).real
    assert abs(ratio - (1 - x ** 6 / 72 + x ** 8 / 576)) < 1e-12
    assert abs(td.taylor_norm_factor(x) - (1 - x ** 6 / 72 + x ** 8 / 576)) < 1e-14


def test_taylor_step_matches_matrix_exponential_to_fifth_order():
    """On a 4^3 cell with one k-point, build h = T + V_x[psi] as a dense matrix and compare the
    Taylor step with expm(-i h dt): the difference is O(dt^5), so halving dt divides it by ~32."""
    grid = (4, 4, 4)
    lattice = inputs.cubic_lattice(5.0)
    kpts = np.array([[0.05, 0.0, -0.03]])
    rng = np.random.default_rng(3)
    psi = inputs.orthonormal_orbitals(rng, grid, lattice, kpts, 2, ecut=50.0)
    occ = np.ones((1, 2))
    A = np.array([0.02, 0.0, 0.0])
    N = 64
    basis = np.eye(N, dtype=complex).reshape(N, *grid)[None]  # [1][N][grid]
    H = td.hamiltonian_apply(psi, occ, basis, kpts, lattice, grid, A, 0.3, 0.25)[0].reshape(N, N).T
    assert np.allclose(H, H.conj().T, atol=1e-12)  # T and V_x are Hermitian
    errs = []
    for dt in (0.1, 0.05):
        ref = (scipy.linalg.expm(-1j * dt * H) @ psi[0].reshape(2, N).T).T.reshape(psi.shape)
        got = td.taylor_step(psi, occ, kpts, lattice, grid, A, 0.3, 0.25, dt)
        errs.append(np.linalg.norm(got - ref))
    assert errs[1] < errs[0] / 20  # fifth-order local error


def test_propagate_uses_vector_potential_of_time():
    grid = (4, 4, 4)
    lattice = inputs.cubic_lattice(5.0)
    kpts = np.zeros((1, 3))
    rng = np.random.default_rng(4)
    psi = inputs.orthonormal_orbitals(rng, grid, lattice, kpts, 1, ecut=50.0)
    occ = np.ones((1, 1))
    E = np.array([0.005, 0.0, 0.0])
    two = td.propagate(psi, occ, kpts, lattice, grid, 0.2, 0.0, 0.02, 2, E)
    s1 = td.taylor_step(psi, occ, kpts, lattice, grid, np.zeros(3), 0.2, 0.0, 0.02)
    s2 = td.taylor_step(s1, occ, kpts, lattice, grid, -E * 0.02, 0.2, 0.0, 0.02)
    np.testing.assert_allclose(two, s2, atol=1e-14)
