"""Pins of the overlap / Gram-Schmidt oracle (cell-normalised orbitals, Sec. II C)."""
import numpy as np

import oracle.ortho as orth
from paper_1507_05156_gb300 import inputs

TRICLINIC = np.array([[7.1, 0.3, -0.4], [0.9, 6.2, 0.5], [-0.6, 1.1, 5.3]])


def _positions(grid, A):
    i1, i2, i3 = np.meshgrid(*(np.arange(n) for n in grid), indexing="ij")
    return (i1[..., None] / grid[0]) * A[0] + (i2[..., None] / grid[1]) * A[1] + (i3[..., None] / grid[2]) * A[2]


def _dv(grid, A):
    return abs(np.linalg.det(A)) / np.prod(grid)


def test_overlap_of_plane_waves_closed_form():
    """Omega^-1/2 e^{iG.r} for distinct G inside the grid's box are orthonormal on the grid:
    dV sum_r e^{i(G_b - G_a).r} / Omega = delta_ab exactly; a scaled copy has overlap c."""
    grid = (6, 5, 4)
    b = 2 * np.pi * np.linalg.inv(TRICLINIC).T
    r = _positions(grid, TRICLINIC)
    Om = abs(np.linalg.det(TRICLINIC))
    ms = [(0, 0, 0), (1, 2, -1), (-2, 1, 1), (2, -2, 0)]
    u = np.stack([np.exp(1j * (r @ (m[0] * b[0] + m[1] * b[1] + m[2] * b[2]))) / np.sqrt(Om) for m in ms])
    S = orth.overlap(u[None], _dv(grid, TRICLINIC))[0]
    np.testing.assert_allclose(S, np.eye(len(ms)), atol=1e-13)
    c = 0.3 - 0.7j
    S2 = orth.overlap(np.stack([u[1], c * u[1]])[None], _dv(grid, TRICLINIC))[0]
    np.testing.assert_allclose(S2, [[1, c], [np.conj(c), abs(c) ** 2]], atol=1e-13)


def test_gram_schmidt_equals_qr_with_positive_diagonal():
    """Orthonormalising columns in order is unique once the triangular factor has a positive
    real diagonal: the result equals numpy's Householder QR of sqrt(dV) u^T with its column
    phases chosen that way (a different algorithm)."""
    grid = (4, 5, 3)
    dV = _dv(grid, TRICLINIC)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((2, 5) + grid) + 1j * rng.standard_normal((2, 5) + grid)
    got = orth.gram_schmidt(u, dV)
    for k in range(2):
        M = np.sqrt(dV) * u[k].reshape(5, -1).T
        Q, R = np.linalg.qr(M)
        ph = np.diag(R) / np.abs(np.diag(R))
        Q = Q * ph[None, :]  # columns with R_aa > 0
        ref = (Q / np.sqrt(dV)).T.reshape((5,) + grid)
        np.testing.assert_allclose(got[k], ref, atol=1e-12)


def test_gram_schmidt_of_orthonormal_set_is_identity_and_result_is_orthonormal():
    grid = (6, 6, 6)
    lattice = inputs.cubic_lattice(inputs.A_SI)
    dV = _dv(grid, lattice)
    kpts = np.array([[0.0, 0.0, 0.0], [0.1, -0.05, 0.2]])
    rng = np.random.default_rng(5)
    u = inputs.orthonormal_orbitals(rng, grid, lattice, kpts, 4, ecut=8.0)
    np.testing.assert_allclose(orth.gram_schmidt(u, dV), u, atol=1e-12)
    v = u + 0.2 * inputs.random_orbitals(9, u.shape) * np.abs(u).mean()
    w = orth.gram_schmidt(v, dV)
    np.testing.assert_allclose(orth.overlap(w, dV), np.broadcast_to(np.eye(4), (2, 4, 4)), atol=1e-12)
    # band 0 only changes by its norm (the order is the band order)
    np.testing.assert_allclose(w[:, 0], v[:, 0] / np.sqrt(orth.overlap(v, dV)[:, 0, 0].real)[:, None, None, None],
                               atol=1e-12)
