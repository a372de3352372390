"""Down-sampled Fock sum on the GPU against the FP64 oracle (Sec. II C, after Eq. "Fock-DS").

The plan takes the indices of the sampled k-points; the orbital arrays keep the full mesh.
Apply, exchange energy and the VJP (including zeros of grad_u_occ at unsampled k-points) are
compared element by element with the oracle's down-sampled form, for the fused complex64
kernels (staged-partner kernel for the target-owner modes, pencil-load kernel for the
occupied-owner VJP) and the complex128 staged form.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_05156_gb300 import hse, inputs

pytestmark = pytest.mark.gpu

TOL = {torch.complex64: 1e-5, torch.complex128: 1e-10}


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def _rel(got, ref):
    got = np.asarray(got, np.complex128)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def _cell(seed, grid, kpts, n_occ, n_tgt, dtype):
    lattice = inputs.cubic_lattice(inputs.A_SI)
    rng = np.random.default_rng(seed)
    rnd = (lambda x: x.astype(np.complex64).astype(np.complex128)) if dtype == torch.complex64 else (lambda x: x)
    u_occ = rnd(inputs.orthonormal_orbitals(rng, grid, lattice, kpts, n_occ, ecut=60.0))
    u_tgt = rnd(inputs.orthonormal_orbitals(rng, grid, lattice, kpts, n_tgt, ecut=60.0))
    ybar = rnd(inputs.random_orbitals(seed + 1, u_tgt.shape) * np.abs(u_tgt).mean())
    occ = rng.random((len(kpts), n_occ)) * 0.5 + 0.5
    return lattice, u_occ, u_tgt, ybar, occ


CASES = [((8, 8, 8), torch.complex64), ((8, 8, 8), torch.complex128), ((20, 20, 20), torch.complex64)]


@pytest.mark.parametrize("grid,dtype", CASES)
def test_downsampled_apply_energy_vjp(grid, dtype):
    lattice = inputs.cubic_lattice(inputs.A_SI)
    rng = np.random.default_rng(7)
    b = 2 * np.pi * np.linalg.inv(lattice).T
    kpts = (rng.random((5, 3)) - 0.5) @ b
    kocc = [3, 0, 4]
    n_occ, n_tgt = 2, 3
    lattice, u_occ, u_tgt, ybar, occ = _cell(11, grid, kpts, n_occ, n_tgt, dtype)
    omega, alpha = inputs.OMEGA, inputs.ALPHA

    plan = hse.Plan(grid, lattice, kpts, n_occ, n_tgt, omega, alpha, dtype=dtype, kocc=kocc)
    out = hse.hse_fock_apply(plan, _dev(u_occ, dtype), _dev(occ, torch.float64), _dev(u_tgt, dtype))
    hse.hse_status(plan)
    ref = oracle.fock_apply(u_occ, occ, u_tgt, kpts, lattice, grid, omega, alpha, kocc=kocc)
    assert _rel(out.cpu().numpy(), ref) <= TOL[dtype]
    # the full-mesh operator differs: the sub-mesh is really used
    full = oracle.fock_apply(u_occ, occ, u_tgt, kpts, lattice, grid, omega, alpha)
    assert _rel(full, ref) > 1e-3

    g_occ, g_tgt, g_om = hse.hse_fock_apply_vjp(plan, _dev(u_occ, dtype), _dev(occ, torch.float64),
                                                _dev(u_tgt, dtype), _dev(ybar, dtype))
    r_occ, r_tgt, r_om = oracle.fock_apply_vjp(u_occ, occ, u_tgt, ybar, kpts, lattice, grid, omega, alpha,
                                               kocc=kocc)
    g_occ = g_occ.cpu().numpy()
    assert _rel(g_tgt.cpu().numpy(), r_tgt) <= TOL[dtype]
    assert _rel(g_occ, r_occ) <= TOL[dtype]
    for k in (1, 2):  # unsampled: exactly zero
        assert np.all(g_occ[k] == 0)
    assert abs(g_om.item() - r_om) <= TOL[dtype] * abs(r_om)

    eplan = hse.Plan(grid, lattice, kpts, n_occ, n_occ, omega, alpha, dtype=dtype, kocc=kocc)
    e = hse.hse_exchange_energy(eplan, _dev(u_occ, dtype), _dev(occ, torch.float64)).item()
    e_ref = oracle.exchange_energy(u_occ, occ, kpts, lattice, grid, omega, alpha, 2.0, kocc=kocc)
    assert e_ref < 0
    assert abs(e - e_ref) <= TOL[dtype] * abs(e_ref)


def test_monkhorst_pack_submesh_sampled_targets():
    """A 6^3 Monkhorst-Pack mesh with the Fock sum over its 2^3 sub-mesh (every third point
    per axis, as the paper's 12^3 -> 4^3), complex64, 8^3 grid; sampled targets against the
    oracle."""
    grid = (8, 8, 8)
    lattice = inputs.cubic_lattice(inputs.A_SI)
    kpts = inputs.monkhorst_pack((6, 6, 6), lattice)
    kocc = inputs.monkhorst_pack_subset((6, 6, 6), (2, 2, 2))
    d = torch.complex64
    lattice, u_occ, u_tgt, ybar, occ = _cell(21, grid, kpts, 2, 2, d)
    plan = hse.Plan(grid, lattice, kpts, 2, 2, inputs.OMEGA, inputs.ALPHA, dtype=d, kocc=kocc)
    out = hse.hse_fock_apply(plan, _dev(u_occ, d), _dev(occ, torch.float64), _dev(u_tgt, d))
    hse.hse_status(plan)
    out = out.cpu().numpy()
    rng = np.random.default_rng(22)
    targets = [(int(k), int(i)) for k, i in zip(rng.integers(0, len(kpts), 6), rng.integers(0, 2, 6))]
    ref = oracle.fock_apply(u_occ, occ, u_tgt, kpts, lattice, grid, inputs.OMEGA, inputs.ALPHA,
                            targets=targets, kocc=kocc)
    got = np.stack([out[k, i] for k, i in targets])
    assert _rel(got, ref) <= 1e-5
