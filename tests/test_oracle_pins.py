"""Pins of the FP64 oracle against the mathematics of Sec. II C (no GPU needed).

Each test checks the oracle against something other than itself: an explicit
O(N^2) sum, a closed form evaluated independently (mpmath or hand-built plane
waves), an invariant the operator must satisfy, or a finite difference.  Together
they catch a dropped term, a wrong sign, a wrong index or a transposed operand in
any step of the oracle.
"""
import json
import os

import mpmath
import numpy as np
import pytest

import oracle
from paper_1507_05156_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# a non-orthogonal cell, so that a transposed reciprocal basis cannot go unnoticed
TRICLINIC = np.array([[7.1, 0.3, -0.4],
                      [0.9, 6.2, 0.5],
                      [-0.6, 1.1, 5.3]])


def _positions(grid, lattice):
    """Cartesian grid points r = i1/N1 a1 + i2/N2 a2 + i3/N3 a3, built here from scratch."""
    i1, i2, i3 = np.meshgrid(*(np.arange(n) for n in grid), indexing="ij")
    A = np.asarray(lattice)
    return (i1[..., None] / grid[0]) * A[0] + (i2[..., None] / grid[1]) * A[1] + (i3[..., None] / grid[2]) * A[2]


def _vtilde_mp(g2, omega):
    """Closed form 4 pi / g^2 (1 - exp(-g^2/(4 omega^2))) in 50-digit arithmetic."""
    mpmath.mp.dps = 50
    g2 = mpmath.mpf(g2)
    w = mpmath.mpf(omega)
    if g2 == 0:
        return float(mpmath.pi / w ** 2)
    return float(4 * mpmath.pi / g2 * (1 - mpmath.exp(-g2 / (4 * w ** 2))))


def _small_cell(seed, grid, kpts, nb, lattice=TRICLINIC):
    rng = np.random.default_rng(seed)
    return inputs.orthonormal_orbitals(rng, grid, lattice, np.asarray(kpts), nb, ecut=40.0)


def test_paper_parameters_fixture():
    with open(os.path.join(GOLDEN, "paper_parameters.json")) as fh:
        p = json.load(fh)
    assert inputs.ALPHA == p["hse_fock_mixing_alpha"]["value"]
    # 0.3 1/angstrom expressed in 1/bohr
    assert abs(inputs.OMEGA_PAPER - p["range_separation_mu_per_angstrom"]["value"] * 0.529177210903) < 1e-12


@pytest.mark.parametrize("grid", [(4, 4, 4), (6, 5, 3), (2, 3, 5)])
def test_forward_transform_equals_direct_sum(grid):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(grid) + 1j * rng.standard_normal(grid)
    np.testing.assert_allclose(oracle.forward_transform(x), oracle.direct_dft(x), rtol=0, atol=1e-13)
    # and the inverse carries no 1/N: inverse(forward(x)) == x
    np.testing.assert_allclose(oracle.inverse_transform(oracle.forward_transform(x)), x, atol=1e-13)


def test_integer_frequencies_match_fftfreq_convention():
    assert list(oracle.integer_frequencies(4)) == [0, 1, -2, -1]
    assert list(oracle.integer_frequencies(5)) == [0, 1, 2, -2, -1]
    assert list(oracle.integer_frequencies(6)) == [0, 1, 2, -3, -2, -1]


def test_g_vectors_are_dual_to_grid_positions():
    grid = (6, 5, 4)
    G = oracle.g_vectors(grid, TRICLINIC)
    r = _positions(grid, TRICLINIC)
    m = np.stack(np.meshgrid(*(oracle.integer_frequencies(n) for n in grid), indexing="ij"), -1)
    idx = np.stack(np.meshgrid(*(np.arange(n) for n in grid), indexing="ij"), -1)
    # G_m . r_i = 2 pi sum_d m_d i_d / N_d  (checked for a few index pairs)
    for a in [(1, 2, 3), (5, 4, 0), (0, 0, 1)]:
        for b in [(2, 1, 1), (3, 4, 2)]:
            lhs = G[a] @ r[b]
            rhs = 2 * np.pi * sum(m[a][d] * idx[b][d] / grid[d] for d in range(3))
            assert abs(lhs - rhs) < 1e-12


@pytest.mark.parametrize("omega", [0.106, inputs.OMEGA_PAPER, 0.7])
def test_screened_kernel_closed_form(omega):
    g2 = np.array([0.0, 1e-14, 1e-8, 1e-3, 0.05, 0.37, 1.0, 4.2, 17.0, 90.0])
    got = oracle.screened_kernel(g2, omega)
    ref = np.array([_vtilde_mp(x, omega) for x in g2])
    np.testing.assert_allclose(got, ref, rtol=2e-15, atol=0)
    assert got[0] == np.pi / omega ** 2


def test_screened_kernel_small_g_series():
    omega = 0.106
    for g in [1e-8, 1e-5, 1e-3]:
        g2 = g * g
        series = np.pi / omega ** 2 - np.pi * g2 / (8 * omega ** 4) + np.pi * g2 ** 2 / (96 * omega ** 6)
        assert abs(oracle.screened_kernel(np.array([g2]), omega)[0] - series) <= 1e-13 * series


def test_screened_kernel_omega_derivative():
    # enough digits that the difference quotient resolves e^{-g^2/4w^2} ~ 1e-58
    mpmath.mp.dps = 160
    for g2 in [0.0, 0.02, 0.9, 6.0]:
        for omega in [0.106, 0.2]:
            f = lambda w: 4 * mpmath.pi / g2 * (1 - mpmath.exp(-g2 / (4 * w ** 2))) if g2 else mpmath.pi / w ** 2
            ref = float(mpmath.diff(f, mpmath.mpf(omega)))
            got = oracle.screened_kernel_domega(np.array([g2]), omega)[0]
            assert abs(got - ref) <= 1e-13 * abs(ref)


def test_plane_wave_closed_form_including_pi_over_omega2_limit():
    """u_i = Omega^-1/2 e^{i G_a r}, u_j = Omega^-1/2 e^{i G_b r}:
    V_x u_i = -alpha f / (N_k Omega) v~(|G_a - G_b + k - k'|) u_i exactly."""
    grid = (6, 5, 4)
    A = TRICLINIC
    Om = abs(np.linalg.det(A))
    b = 2 * np.pi * np.linalg.inv(A).T
    r = _positions(grid, A)
    kpts = np.array([[0.05, -0.11, 0.02], [-0.2, 0.07, 0.13]])
    omega, alpha = 0.31, 0.25

    def pw(m):
        G = m[0] * b[0] + m[1] * b[1] + m[2] * b[2]
        return np.exp(1j * (r @ G)) / np.sqrt(Om), G

    cases = [((1, 2, -1), (1, 2, -1), 0, 0),    # same G and same k: the pi/omega^2 limit
             ((1, 2, -1), (1, 2, -1), 0, 1),    # same G, q != 0
             ((2, -1, 1), (0, 1, 0), 1, 0)]     # G_a != G_b, q != 0
    for ma, mb, k, kp in cases:
        ua, Ga = pw(ma)
        ub, Gb = pw(mb)
        u_tgt = np.zeros((2, 1) + grid, complex)
        u_occ = np.zeros((2, 1) + grid, complex)
        u_tgt[k, 0] = ua
        u_occ[kp, 0] = ub
        f = 0.7
        occ = np.zeros((2, 1))
        occ[kp, 0] = f
        out = oracle.fock_apply(u_occ, occ, u_tgt, kpts, A, grid, omega, alpha)
        q = kpts[k] - kpts[kp]
        g = Ga - Gb + q
        v = _vtilde_mp(float(g @ g), omega)
        expect = -alpha * f / (2 * Om) * v * ua
        np.testing.assert_allclose(out[k, 0], expect, rtol=0, atol=1e-13 * np.abs(expect).max())
        if ma == mb and k == kp:
            assert abs(v - np.pi / omega ** 2) < 1e-12


def test_fft_form_equals_realspace_double_sum():
    grid = (4, 3, 5)
    kpts = np.array([[0.0, 0.0, 0.0], [0.21, -0.13, 0.08]])
    u_occ = _small_cell(3, grid, kpts, 2)
    u_tgt = _small_cell(4, grid, kpts, 3)
    occ = np.array([[1.0, 0.6], [0.9, 0.3]])
    a = oracle.fock_apply(u_occ, occ, u_tgt, kpts, TRICLINIC, grid, 0.23, 0.25)
    b = oracle.fock_apply_realspace(u_occ, occ, u_tgt, kpts, TRICLINIC, grid, 0.23, 0.25)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * np.abs(b).max())


def test_constant_kernel_limit_is_a_local_product():
    """For omega -> infinity v~ -> pi/omega^2 (1 - g^2/(8 omega^2)), so K_q becomes
    (pi/omega^2) times the identity and V_x u_i -> -alpha pi/(omega^2 N_k) sum f |u_j|^2 u_i."""
    grid = (5, 4, 6)
    kpts = np.array([[0.0, 0.0, 0.0], [0.1, 0.2, -0.1], [-0.3, 0.05, 0.0]])
    u_occ = _small_cell(5, grid, kpts, 2)
    u_tgt = _small_cell(6, grid, kpts, 2)
    occ = np.array([[1.0, 0.5], [1.0, 1.0], [0.2, 0.9]])
    omega = 2.0e4
    out = oracle.fock_apply(u_occ, occ, u_tgt, kpts, TRICLINIC, grid, omega, 0.25)
    dens = np.einsum("kj,kj...->...", occ, np.abs(u_occ) ** 2)
    expect = -0.25 * np.pi / (omega ** 2 * 3) * dens[None, None] * u_tgt
    np.testing.assert_allclose(out, expect, rtol=0, atol=1e-8 * np.abs(expect).max())


def test_hermitian_and_negative_semidefinite():
    grid = (6, 4, 5)
    kpts = np.array([[0.0, 0.0, 0.0], [0.17, 0.0, -0.09]])
    u_occ = _small_cell(7, grid, kpts, 3)
    occ = np.ones((2, 3))
    ab = inputs.random_orbitals(8, (2, 2) + grid)
    v = oracle.fock_apply(u_occ, occ, ab, kpts, TRICLINIC, grid, 0.106, 0.25)
    for k in range(2):
        a, b_ = ab[k, 0], ab[k, 1]
        va, vb = v[k, 0], v[k, 1]
        lhs = np.vdot(a, vb)
        rhs = np.conj(np.vdot(b_, va))
        assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
        assert np.vdot(a, va).real < 0 and np.vdot(b_, vb).real < 0


def test_exchange_energy_negative_and_gradient_by_finite_difference():
    # Odd axes: the G-set is then symmetric under G -> -G, so conj(K_q) = K_{-q} and
    # E_x is exactly the functional whose gradient is V_x.  On an even axis the
    # Nyquist plane (m = -N/2 only) breaks that symmetry and the identity holds up
    # to the Nyquist components.
    grid = (5, 3, 5)
    kpts = np.array([[0.0, 0.0, 0.0], [0.2, 0.1, 0.0]])
    u = _small_cell(9, grid, kpts, 2)
    occ = np.array([[1.0, 0.8], [0.6, 1.0]])
    omega, alpha, gs = 0.15, 0.25, 2.0
    E = oracle.exchange_energy(u, occ, kpts, TRICLINIC, grid, omega, alpha, gs)
    assert E < 0
    d = inputs.random_orbitals(10, u.shape) * np.abs(u).mean()   # same scale as u
    eps = 1e-5
    Ep = oracle.exchange_energy(u + eps * d, occ, kpts, TRICLINIC, grid, omega, alpha, gs)
    Em = oracle.exchange_energy(u - eps * d, occ, kpts, TRICLINIC, grid, omega, alpha, gs)
    fd = (Ep - Em) / (2 * eps)
    vx = oracle.fock_apply(u, occ, u, kpts, TRICLINIC, grid, omega, alpha)
    dV = oracle.cell_volume(TRICLINIC) / np.prod(grid)
    nk = len(kpts)
    an = 2 * gs * dV / nk * sum(occ[k, i] * np.vdot(d[k, i], vx[k, i]).real for k in range(2) for i in range(2))
    assert abs(fd - an) <= 1e-8 * abs(an)


def test_supercell_at_gamma_equals_primitive_cell_with_two_kpoints():
    """A 2x1x1 supercell at Gamma holding e^{ik.r} u_{b,k}/sqrt(2) for k in {0, b1/2}
    gives V' psi'_i = e^{ik.r} (V_x u)_{i,k} / sqrt(2): pins q = k - k' and 1/N_k.

    The orbitals are band-limited to |m1| <= 1 along b1, so every pair density and
    every G + q stays inside both the primitive and the supercell FFT boxes (q is
    not folded, reading 4), and the identity is exact.
    """
    A = TRICLINIC
    b = 2 * np.pi * np.linalg.inv(A).T
    g = (8, 3, 4)
    kpts = np.array([np.zeros(3), 0.5 * b[0]])
    rng = np.random.default_rng(11)
    coef = np.zeros((2, 2) + g, complex)
    for m1 in (-1, 0, 1):
        coef[:, :, m1] = rng.standard_normal((2, 2) + g[1:]) + 1j * rng.standard_normal((2, 2) + g[1:])
    dV = abs(np.linalg.det(A)) / np.prod(g)
    u = inputs.gram_schmidt(np.fft.ifftn(coef, axes=(2, 3, 4)), dV)
    occ = np.ones((2, 2))
    omega, alpha = 0.2, 0.25
    v = oracle.fock_apply(u, occ, u, kpts, A, g, omega, alpha)
    As = A.copy()
    As[0] = 2 * A[0]
    gs_ = (16, 3, 4)
    rs = _positions(gs_, As)
    psi = np.zeros((1, 4) + gs_, complex)
    expect = np.zeros_like(psi)
    for k in range(2):
        ph = np.exp(1j * (rs @ kpts[k]))
        for bnd in range(2):
            psi[0, 2 * k + bnd] = ph * np.tile(u[k, bnd], (2, 1, 1)) / np.sqrt(2)
            expect[0, 2 * k + bnd] = ph * np.tile(v[k, bnd], (2, 1, 1)) / np.sqrt(2)
    vs = oracle.fock_apply(psi, np.ones((1, 4)), psi, np.zeros((1, 3)), As, gs_, omega, alpha)
    np.testing.assert_allclose(vs, expect, rtol=0, atol=1e-12 * np.abs(expect).max())


def test_vjp_matches_central_finite_differences():
    grid = (4, 4, 3)
    kpts = np.array([[0.0, 0.0, 0.0], [0.15, -0.1, 0.2]])
    u_occ = _small_cell(12, grid, kpts, 2)
    u_tgt = _small_cell(13, grid, kpts, 3)
    occ = np.array([[1.0, 0.7], [0.4, 1.0]])
    omega, alpha = 0.25, 0.25
    w = inputs.random_orbitals(14, u_tgt.shape)

    def L(uo, ut, om):
        y = oracle.fock_apply(uo, occ, ut, kpts, TRICLINIC, grid, om, alpha)
        return np.real(np.vdot(w, y))

    g_occ, g_tgt, g_om = oracle.fock_apply_vjp(u_occ, occ, u_tgt, w, kpts, TRICLINIC, grid, omega, alpha)
    h = 1e-5
    d_occ = inputs.random_orbitals(15, u_occ.shape)
    d_tgt = inputs.random_orbitals(16, u_tgt.shape)
    fd = (L(u_occ + h * d_occ, u_tgt, omega) - L(u_occ - h * d_occ, u_tgt, omega)) / (2 * h)
    an = np.real(np.vdot(g_occ, d_occ))
    assert abs(fd - an) <= 1e-7 * abs(an)
    fd = (L(u_occ, u_tgt + h * d_tgt, omega) - L(u_occ, u_tgt - h * d_tgt, omega)) / (2 * h)
    an = np.real(np.vdot(g_tgt, d_tgt))
    assert abs(fd - an) <= 1e-7 * abs(an)
    fd = (L(u_occ, u_tgt, omega + h) - L(u_occ, u_tgt, omega - h)) / (2 * h)
    assert abs(fd - g_om) <= 1e-7 * abs(g_om)


def test_monkhorst_pack_mesh():
    A = inputs.cubic_lattice(10.26)
    b = 2 * np.pi / 10.26
    k = inputs.monkhorst_pack((2, 2, 2), A)
    assert k.shape == (8, 3)
    np.testing.assert_allclose(np.unique(np.round(k / b, 12)), [-0.25, 0.25])
    k3 = inputs.monkhorst_pack((3, 3, 3), A)
    np.testing.assert_allclose(np.unique(np.round(k3 / b, 12)), [-1 / 3, 0.0, 1 / 3])


def test_generated_orbitals_orthonormal():
    c = inputs.workload(0)
    dV = oracle.cell_volume(c.lattice) / c.npts
    u = c.u_occ.reshape(c.nk, c.n_occ, -1)
    S = dV * np.einsum("kan,kbn->kab", u.conj(), u)
    np.testing.assert_allclose(S, np.broadcast_to(np.eye(c.n_occ), S.shape), atol=1e-12)


# ---------------------------------------------------------------------------
# Down-sampled Fock sum (Sec. II C after Eq. "Fock-DS"): k' over a q-point sub-mesh, 1/N_q
# ---------------------------------------------------------------------------

def test_monkhorst_pack_submesh_is_a_subset():
    A = TRICLINIC
    for n, m in (((12, 12, 12), (4, 4, 4)), ((6, 3, 9), (2, 1, 3)), ((3, 3, 3), (1, 1, 1))):
        idx = inputs.monkhorst_pack_subset(n, m)
        np.testing.assert_allclose(inputs.monkhorst_pack(n, A)[idx], inputs.monkhorst_pack(m, A), atol=1e-13)
    with pytest.raises(ValueError):
        inputs.monkhorst_pack_subset((4, 4, 4), (2, 2, 2))  # even factor: not a subset


def test_downsampled_plane_wave_closed_form():
    """One plane wave per k-point: V_x u_i = -alpha/(N_q Omega) sum_{k' in S} f_k' v~(|G_a - G_b + k - k'|) u_i,
    evaluated term by term in 50-digit arithmetic, for a strict sub-mesh S with unequal f."""
    grid = (5, 4, 6)
    A = TRICLINIC
    Om = abs(np.linalg.det(A))
    b = 2 * np.pi * np.linalg.inv(A).T
    r = _positions(grid, A)
    kpts = np.array([[0.05, -0.11, 0.02], [-0.2, 0.07, 0.13], [0.11, 0.16, -0.09], [0.0, -0.05, 0.21]])
    omega, alpha = 0.23, 0.25
    Ga = 1 * b[0] - 1 * b[1] + 1 * b[2]   # G_a - G_b = (1, -1, 2): inside the 5 x 4 x 6 box
    Gb = 0 * b[0] + 0 * b[1] - 1 * b[2]
    ua = np.exp(1j * (r @ Ga)) / np.sqrt(Om)
    ub = np.exp(1j * (r @ Gb)) / np.sqrt(Om)
    u_tgt = np.broadcast_to(ua, (4, 1) + grid).copy()
    u_occ = np.broadcast_to(ub, (4, 1) + grid).copy()
    occ = np.array([[0.9], [0.3], [0.6], [1.0]])
    kocc = [3, 1, 2]
    out = oracle.fock_apply(u_occ, occ, u_tgt, kpts, A, grid, omega, alpha, kocc=kocc)
    for k in range(4):
        s = 0.0
        for kp in kocc:
            g = Ga - Gb + kpts[k] - kpts[kp]
            s += occ[kp, 0] * _vtilde_mp(float(g @ g), omega)
        expect = -alpha / (len(kocc) * Om) * s * ua
        np.testing.assert_allclose(out[k, 0], expect, rtol=0, atol=1e-13 * np.abs(expect).max())


def test_downsampled_fft_form_equals_realspace_double_sum():
    grid = (3, 4, 3)
    kpts = np.array([[0.0, 0.0, 0.0], [0.21, -0.1, 0.05], [-0.13, 0.17, 0.09]])
    u_occ = _small_cell(41, grid, kpts, 2)
    u_tgt = _small_cell(42, grid, kpts, 2)
    occ = np.array([[1.0, 0.5], [0.8, 0.2], [0.3, 1.0]])
    kocc = [2, 0]
    a = oracle.fock_apply(u_occ, occ, u_tgt, kpts, TRICLINIC, grid, 0.27, 0.25, kocc=kocc)
    b = oracle.fock_apply_realspace(u_occ, occ, u_tgt, kpts, TRICLINIC, grid, 0.27, 0.25, kocc=kocc)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    # the full sub-mesh is the undown-sampled operator
    full = oracle.fock_apply(u_occ, occ, u_tgt, kpts, TRICLINIC, grid, 0.27, 0.25)
    np.testing.assert_array_equal(oracle.fock_apply(u_occ, occ, u_tgt, kpts, TRICLINIC, grid, 0.27, 0.25,
                                                    kocc=[0, 1, 2]), full)


def test_downsampled_hermitian_negative_and_vjp_by_finite_differences():
    grid = (4, 3, 4)
    kpts = np.array([[0.0, 0.0, 0.0], [0.15, -0.1, 0.2], [-0.07, 0.12, -0.16]])
    kocc = [1, 2]
    u_occ = _small_cell(51, grid, kpts, 2)
    occ = np.array([[1.0, 0.7], [0.4, 1.0], [0.9, 0.6]])
    omega, alpha = 0.25, 0.25
    # Hermitian and negative semidefinite at each k (the occupied set is fixed)
    a = inputs.random_orbitals(52, (3, 1) + grid)
    bb = inputs.random_orbitals(53, (3, 1) + grid)
    va = oracle.fock_apply(u_occ, occ, a, kpts, TRICLINIC, grid, omega, alpha, kocc=kocc)
    vb = oracle.fock_apply(u_occ, occ, bb, kpts, TRICLINIC, grid, omega, alpha, kocc=kocc)
    for k in range(3):
        ab, ba = np.vdot(a[k], vb[k]), np.vdot(bb[k], va[k])
        assert abs(ab - np.conj(ba)) <= 1e-13 * abs(ab)
        assert np.vdot(a[k], va[k]).real < 0
    # VJP against central differences; no gradient reaches the unsampled k-point
    u_tgt = _small_cell(54, grid, kpts, 2)
    w = inputs.random_orbitals(55, u_tgt.shape)

    def L(uo, ut, om):
        return np.real(np.vdot(w, oracle.fock_apply(uo, occ, ut, kpts, TRICLINIC, grid, om, alpha, kocc=kocc)))

    g_occ, g_tgt, g_om = oracle.fock_apply_vjp(u_occ, occ, u_tgt, w, kpts, TRICLINIC, grid, omega, alpha,
                                               kocc=kocc)
    assert np.all(g_occ[0] == 0)
    h = 1e-5
    for seed, (g, arg) in enumerate(((g_occ, 0), (g_tgt, 1))):
        d = inputs.random_orbitals(56 + seed, g.shape)
        args_p = [u_occ, u_tgt]
        args_m = [u_occ, u_tgt]
        args_p[arg] = args_p[arg] + h * d
        args_m[arg] = args_m[arg] - h * d
        fd = (L(args_p[0], args_p[1], omega) - L(args_m[0], args_m[1], omega)) / (2 * h)
        an = np.real(np.vdot(g, d))
        assert abs(fd - an) <= 1e-7 * abs(an)
    fd = (L(u_occ, u_tgt, omega + h) - L(u_occ, u_tgt, omega - h)) / (2 * h)
    assert abs(fd - g_om) <= 1e-7 * abs(g_om)
    # E_x with a down-sampled Fock sum is still negative
    assert oracle.exchange_energy(u_occ, occ, kpts, TRICLINIC, grid, omega, alpha, kocc=kocc) < 0
