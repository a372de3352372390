"""FP64 overlap matrices and Gram-Schmidt orthonormalisation on the GPU against the FP64 oracle
(cell-normalised orbitals; the propagator check of Sec. II C)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_05156_gb300 import hse, inputs

pytestmark = pytest.mark.gpu


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def _setup(n, nk, nb, dtype, seed):
    grid = (n, n, n)
    lattice = inputs.cubic_lattice(inputs.A_SI)
    dV = abs(np.linalg.det(lattice)) / n ** 3
    rng = np.random.default_rng(seed)
    b = 2 * np.pi * np.linalg.inv(lattice).T
    kpts = (rng.random((nk, 3)) - 0.5) @ b
    u = inputs.random_orbitals(seed, (nk, nb) + grid) / np.sqrt(abs(np.linalg.det(lattice)))
    if dtype == torch.complex64:
        u = u.astype(np.complex64).astype(np.complex128)
    plan = hse.Plan(grid, lattice, kpts, nb, nb, inputs.OMEGA, inputs.ALPHA, dtype=dtype)
    return plan, u, dV


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_overlap_matches_oracle(dtype):
    plan, u, dV = _setup(8, 3, 5, dtype, 11)
    S = hse.hse_overlap(plan, _dev(u, dtype)).cpu().numpy()
    ref = oracle.ortho.overlap(u, dV)
    assert np.abs(S - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(S - np.conj(np.transpose(S, (0, 2, 1)))).max() == 0.0  # written Hermitian


@pytest.mark.parametrize("n,nk,nb,dtype", [(8, 3, 5, torch.complex128), (8, 3, 5, torch.complex64),
                                           (24, 2, 32, torch.complex128), (24, 2, 32, torch.complex64)])
def test_orthonormalize_matches_oracle(n, nk, nb, dtype):
    plan, u, dV = _setup(n, nk, nb, dtype, 20 + n)
    d = _dev(u, dtype)
    hse.hse_orthonormalize(plan, d)
    hse.hse_status(plan)
    ref = oracle.ortho.gram_schmidt(u, dV)
    got = d.cpu().numpy().astype(np.complex128)
    tol = 1e-12 if dtype == torch.complex128 else 1e-6  # complex64: FP64 arithmetic, one rounding
    err = np.linalg.norm((got - ref).reshape(nk * nb, -1), axis=1) / np.linalg.norm(ref.reshape(nk * nb, -1), axis=1)
    assert err.max() <= tol
    S = hse.hse_overlap(plan, d).cpu().numpy()
    assert np.abs(S - np.eye(nb)[None]).max() <= (1e-13 if dtype == torch.complex128 else 2e-6)


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_linearly_dependent_band_is_reported(dtype):
    plan, u, dV = _setup(8, 2, 4, dtype, 5)
    u[1, 2] = (0.5 - 0.25j) * u[1, 0] + 2.0 * u[1, 1]  # band 2 of k-point 1 is in the span
    if dtype == torch.complex64:
        u = u.astype(np.complex64).astype(np.complex128)
    d = _dev(u, dtype)
    hse.hse_orthonormalize(plan, d)
    with pytest.raises(hse.HseError) as e:
        hse.hse_status(plan)
    assert e.value.code == -8
    got = d.cpu().numpy()
    assert np.all(got[1, 2] == 0)
    ref = oracle.ortho.gram_schmidt(u[:1], dV)  # k-point 0 is untouched by the failure
    assert np.abs(got[0] - ref[0]).max() <= (1e-12 if dtype == torch.complex128 else 1e-6) * np.abs(ref).max()
    hse.hse_status(plan)  # the status word was cleared
