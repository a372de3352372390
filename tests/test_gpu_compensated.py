"""Compensated accumulation over k' (Sec. II C, Eq. "Fock": V_x u sums the pair terms over
every k' and occupied band).

A k-mesh of N_k copies of one k-point with identical orbitals makes every pair term of a
target the same FP32 value; the 1/N_k of the Fock sum cancels the N_k copies, so the exact
operator is the one-k-point operator, which the FP64 oracle computes directly.  Summed in
plain FP32, N_k = 512 equal terms drift by a few 1e-6 relative (the rounding of each addition
has the same sign); the compensated sums stay at the rounding of a single pair term (~1e-7).
The same holds for the VJP with respect to the occupied orbitals, whose sum runs over the
target k-points, on the pencil-load kernel, and for the 24^3 grid.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_05156_gb300 import hse, inputs

pytestmark = pytest.mark.gpu

NK = 512
TOL = 4e-7


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def _copies(n, n_occ, n_tgt, seed):
    grid = (n, n, n)
    lattice = inputs.cubic_lattice(inputs.A_SI)
    rng = np.random.default_rng(seed)
    b = 2 * np.pi * np.linalg.inv(lattice).T
    k0 = ((rng.random(3) - 0.5) @ b)[None, :]
    c64 = lambda x: np.ascontiguousarray(x).astype(np.complex64).astype(np.complex128)
    u_occ1 = c64(inputs.orthonormal_orbitals(rng, grid, lattice, k0, n_occ, ecut=60.0))
    u_tgt1 = c64(inputs.orthonormal_orbitals(rng, grid, lattice, k0, n_tgt, ecut=60.0))
    ybar1 = c64(inputs.random_orbitals(seed + 1, u_tgt1.shape) * np.abs(u_tgt1).mean())
    occ1 = rng.random((1, n_occ)) * 0.5 + 0.5
    rep = lambda x: np.repeat(x, NK, axis=0)
    return grid, lattice, k0, u_occ1, u_tgt1, ybar1, occ1, rep(k0), rep(u_occ1), rep(u_tgt1), rep(ybar1), rep(occ1)


def _max_rel(got, ref1):
    """Largest relative error of any of the NK copies against the one-k-point result."""
    got = np.asarray(got, np.complex128)
    return max(float(np.linalg.norm(got[k] - ref1[0]) / np.linalg.norm(ref1[0])) for k in range(NK))


@pytest.mark.parametrize("n", [8, 24])
def test_apply_sum_over_copies(n):
    grid, lattice, k0, u_occ1, u_tgt1, _, occ1, kpts, u_occ, u_tgt, _, occ = _copies(n, 2, 1, 40 + n)
    omega, alpha = inputs.OMEGA, inputs.ALPHA
    d = torch.complex64
    plan = hse.Plan(grid, lattice, kpts, 2, 1, omega, alpha, dtype=d)
    out = hse.hse_fock_apply(plan, _dev(u_occ, d), _dev(occ, torch.float64), _dev(u_tgt, d))
    hse.hse_status(plan)
    ref1 = oracle.fock_apply(u_occ1, occ1, u_tgt1, k0, lattice, grid, omega, alpha)
    assert _max_rel(out.cpu().numpy(), ref1) <= TOL


def test_vjp_occ_sum_over_copies():
    n = 8
    grid, lattice, k0, u_occ1, u_tgt1, ybar1, occ1, kpts, u_occ, u_tgt, ybar, occ = _copies(n, 1, 2, 77)
    omega, alpha = inputs.OMEGA, inputs.ALPHA
    d = torch.complex64
    plan = hse.Plan(grid, lattice, kpts, 1, 2, omega, alpha, dtype=d)
    g_occ, _, _ = hse.hse_fock_apply_vjp(plan, _dev(u_occ, d), _dev(occ, torch.float64), _dev(u_tgt, d),
                                         _dev(ybar, d), need_tgt=False, need_omega=False)
    hse.hse_status(plan)
    r_occ, _, _ = oracle.fock_apply_vjp(u_occ1, occ1, u_tgt1, ybar1, k0, lattice, grid, omega, alpha)
    assert _max_rel(g_occ.cpu().numpy(), r_occ) <= TOL
