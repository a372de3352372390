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


def test_hamiltonian_on_plane_wave_with_local_potential_closed_form():
    """alpha = 0: h = T[A] + v_loc (Sec. II A, Eq. "tdks-h"), so on a plane wave u = e^{iG.r}
    and v_loc(r) = c + d cos(G1.r), built here from the grid positions,
    h u = (1/2 |G + k + A|^2 + c + d cos(G1.r)) u point by point."""
    grid = (6, 5, 4)
    b = 2 * np.pi * np.linalg.inv(TRICLINIC).T
    r = _positions(grid, TRICLINIC)
    G = 1 * b[0] + 2 * b[1] - 1 * b[2]
    G1 = 2 * b[0] - 1 * b[2]
    u = np.exp(1j * (r @ G))[None, None]
    k = np.array([[0.07, 0.12, -0.04]])
    A = np.array([-0.01, 0.02, 0.03])
    c, d = 0.35, -0.8
    vloc = c + d * np.cos(r @ G1)
    out = td.hamiltonian_apply(u, np.ones((1, 1)), u, k, TRICLINIC, grid, A, 0.2, 0.0, vloc)
    g = G + k[0] + A
    np.testing.assert_allclose(out, (0.5 * (g @ g) + vloc) * u, atol=1e-12)


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


# ---------------------------------------------------------------------------
# Current (Eqs. current_dns / current_elec) and the laser-pulse driver (Sec. IV / V)
# ---------------------------------------------------------------------------

def test_current_of_plane_waves_closed_form():
    """One plane wave Omega^-1/2 e^{iG_k r} per k-point: J = -sum_k g_s f_k / (N_k Omega) (G_k + k + A)."""
    grid = (5, 4, 6)
    A_ = TRICLINIC
    Om = abs(np.linalg.det(A_))
    b = 2 * np.pi * np.linalg.inv(A_).T
    r = _positions(grid, A_)
    kpts = np.array([[0.05, -0.11, 0.02], [-0.2, 0.07, 0.13]])
    ms = [(1, -1, 2), (-2, 1, 0)]
    u = np.zeros((2, 1) + grid, complex)
    Gs = []
    for k, m in enumerate(ms):
        G = m[0] * b[0] + m[1] * b[1] + m[2] * b[2]
        Gs.append(G)
        u[k, 0] = np.exp(1j * (r @ G)) / np.sqrt(Om)
    occ = np.array([[0.7], [0.4]])
    A = np.array([0.03, -0.01, 0.02])
    J = td.current(u, occ, kpts, A_, grid, A, spin_degeneracy=2.0)
    expect = -sum(2.0 * occ[k, 0] / (2 * Om) * (Gs[k] + kpts[k] + A) for k in range(2))
    np.testing.assert_allclose(J, expect, rtol=0, atol=1e-14 * np.abs(expect).max())


def test_current_diamagnetic_shift_and_zero_for_real_orbitals():
    """J(A') - J(A) = -(g_s / (N_k Omega)) sum f (A' - A) for normalised orbitals; real orbitals at
    k = 0 on an odd grid (every G has its -G) carry no current at A = 0."""
    grid = (5, 3, 5)
    kpts = np.array([[0.0, 0.0, 0.0], [0.1, 0.05, -0.08]])
    rng = np.random.default_rng(9)
    u = inputs.orthonormal_orbitals(rng, grid, TRICLINIC, kpts, 3, ecut=30.0)
    occ = np.array([[1.0, 0.6, 0.2], [0.9, 0.5, 0.1]])
    Om = abs(np.linalg.det(TRICLINIC))
    A0, A1 = np.array([0.01, 0.0, -0.02]), np.array([-0.04, 0.03, 0.01])
    d = td.current(u, occ, kpts, TRICLINIC, grid, A1) - td.current(u, occ, kpts, TRICLINIC, grid, A0)
    np.testing.assert_allclose(d, -2.0 / (2 * Om) * occ.sum() * (A1 - A0), rtol=1e-12, atol=0)
    ur = np.real(u[:1]).astype(complex)
    ur /= np.sqrt(np.sum(np.abs(ur) ** 2, axis=(2, 3, 4), keepdims=True) * Om / np.prod(grid))
    J = td.current(ur, np.ones((1, 3)), kpts[:1], TRICLINIC, grid, np.zeros(3))
    assert np.abs(J).max() < 1e-15


def test_pulse_field_is_minus_dA_dt_and_vanishes_outside():
    E0, w, Td, d = 0.01, 0.057, 400.0, (0.0, 0.0, 1.0)
    for t in (13.0, 101.7, 250.2, 399.0):
        h = 1e-4
        num = -(td.pulse_vector_potential(t + h, E0, w, Td, d) - td.pulse_vector_potential(t - h, E0, w, Td, d)) / (2 * h)
        np.testing.assert_allclose(td.pulse_field(t, E0, w, Td, d), num, rtol=1e-7, atol=1e-12)
    for t in (-1.0, 0.0, Td, Td + 5):
        assert np.all(td.pulse_vector_potential(t, E0, w, Td, d) == 0)
        assert np.all(td.pulse_field(t, E0, w, Td, d) == 0)


def test_pulse_on_free_plane_wave_work_closed_form():
    """alpha = 0, one plane wave: it stays an eigenvector of h(t_s) with eps_s = |G + k + A_s|^2 / 2,
    so each step multiplies its norm by the truncated-series factor F(eps_s dt) and
    J_s = -c (G + k + A_s) prod_{j<s} F(eps_j dt), c = g_s f / (N_k Omega).  The work
    W(t) = int J . E = c [(G + k) . A + |A|^2 / 2]_0^t (E = -dA/dt) is followed by the trapezoidal
    W to O(dt^2) and returns to 0 after the pulse."""
    grid = (4, 4, 4)
    A_ = inputs.cubic_lattice(6.0)
    Om = 6.0 ** 3
    b = 2 * np.pi / 6.0
    G = np.array([b, 0.0, -b])
    u = np.exp(1j * (_positions(grid, A_) @ G))[None, None] / np.sqrt(Om)
    k = np.array([[0.02, 0.0, 0.01]])
    E0, w, Td, d = 0.02, 0.4, 40.0, (1.0, 0.0, 0.0)
    dt, nsteps = 0.05, 900
    psi, J, W = td.propagate_pulse(u, np.ones((1, 1)), k, A_, grid, 0.2, 0.0, dt, nsteps, E0, w, Td, d)
    c = 2.0 / Om
    # trapezoidal-rule error bound dt^2 / 12 * T_d * max |(J . E)''|, with
    # |(J . E)''| <= c E0 (|G + k| + E0 / w) (w + 2 pi / T_d)^2
    tol = dt ** 2 / 12 * Td * c * E0 * (np.abs(G + k[0]).max() + E0 / w) * (w + 2 * np.pi / Td) ** 2
    norm = 1.0
    for s in range(nsteps + 1):
        A = td.pulse_vector_potential(s * dt, E0, w, Td, d)
        gk = G + k[0] + A
        if s % 150 == 0:
            np.testing.assert_allclose(J[s], -c * gk * norm, rtol=1e-12, atol=1e-15)
            Wex = c * ((G + k[0]) @ A + 0.5 * A @ A)
            assert abs(W[s] - Wex) <= tol
        norm *= td.taylor_norm_factor(0.5 * (gk @ gk) * dt)
    assert abs(W[-1]) <= tol


# ---------------------------------------------------------------------------
# Hartree potential (Sec. II A Eq. tdks-h, Sec. V Eq. Eex01)
# ---------------------------------------------------------------------------

def test_hartree_of_two_plane_waves_closed_form():
    """u = (e^{iG1 r} + e^{iG2 r}) / sqrt(2 Omega): rho = c (1 + cos(dG . r)), c = g_s f / (N_k Omega), so
    v_H = 4 pi c cos(dG . r) / |dG|^2 exactly (dG inside the box), and E_H = 1/2 Omega c^2 4 pi / |dG|^2 / 2."""
    grid = (6, 5, 8)
    A_ = TRICLINIC
    Om = abs(np.linalg.det(A_))
    b = 2 * np.pi * np.linalg.inv(A_).T
    r = _positions(grid, A_)
    G1 = 1 * b[0] - 1 * b[1] + 2 * b[2]
    G2 = 0 * b[0] + 1 * b[1] + 1 * b[2]
    u = ((np.exp(1j * (r @ G1)) + np.exp(1j * (r @ G2))) / np.sqrt(2 * Om))[None, None]
    f = 0.8
    c = 2.0 * f / Om
    dG = G1 - G2
    vh = td.hartree_potential(u, np.array([[f]]), A_, grid)
    expect = 4 * np.pi * c * np.cos(r @ dG) / (dG @ dG)
    np.testing.assert_allclose(vh, expect, rtol=0, atol=1e-13 * np.abs(expect).max())
    eh = td.hartree_energy(u, np.array([[f]]), A_, grid)
    assert abs(eh - 0.5 * Om * c * c * 4 * np.pi / (dG @ dG) / 2) <= 1e-13 * eh


def test_hartree_of_uniform_density_vanishes_and_energy_is_nonnegative():
    grid = (4, 5, 3)
    kpts = np.array([[0.0, 0.0, 0.0], [0.1, -0.05, 0.2]])
    A_ = TRICLINIC
    Om = abs(np.linalg.det(A_))
    b = 2 * np.pi * np.linalg.inv(A_).T
    r = _positions(grid, A_)
    G = 1 * b[0] + 1 * b[2]
    u = np.exp(1j * (r @ G))[None, None].repeat(2, axis=0) / np.sqrt(Om)
    assert np.abs(td.hartree_potential(u, np.ones((2, 1)), A_, grid)).max() < 1e-14
    rng = np.random.default_rng(5)
    w = inputs.orthonormal_orbitals(rng, grid, A_, kpts, 3, ecut=40.0)
    occ = np.array([[1.0, 0.5, 0.2], [0.9, 0.4, 0.0]])
    assert td.hartree_energy(w, occ, A_, grid) > 0
    # charge: the density integrates to g_s sum f / N_k electrons per cell
    rho = td.density(w, occ, grid)
    assert abs(rho.sum() * Om / np.prod(grid) - 2.0 * occ.sum() / 2) < 1e-12


def test_taylor_step_with_local_potential_matches_matrix_exponential():
    """With a random real local potential added, h stays Hermitian and the Taylor step keeps its
    fifth-order local error against expm(-i h dt) (halving dt divides it by ~32)."""
    grid = (4, 4, 4)
    lattice = inputs.cubic_lattice(5.0)
    kpts = np.array([[0.05, 0.0, -0.03]])
    rng = np.random.default_rng(7)
    psi = inputs.orthonormal_orbitals(rng, grid, lattice, kpts, 2, ecut=50.0)
    occ = np.ones((1, 2))
    A = np.array([0.02, 0.0, 0.0])
    vloc = rng.standard_normal(grid) * 0.3
    N = 64
    basis = np.eye(N, dtype=complex).reshape(N, *grid)[None]
    H = td.hamiltonian_apply(psi, occ, basis, kpts, lattice, grid, A, 0.3, 0.25, vloc)[0].reshape(N, N).T
    assert np.allclose(H, H.conj().T, atol=1e-12)
    errs = []
    for dt in (0.1, 0.05):
        ref = (scipy.linalg.expm(-1j * dt * H) @ psi[0].reshape(2, N).T).T.reshape(psi.shape)
        got = td.taylor_step(psi, occ, kpts, lattice, grid, A, 0.3, 0.25, dt, vloc=vloc)
        errs.append(np.linalg.norm(got - ref))
    assert errs[1] < errs[0] / 20
