"""Each pencil layout of the fused kernels against the FP64 oracle.

The layout is chosen per plan through HSE_BLOCKS_PER_SM: for the staged-partner kernel -1 two
pencils per thread, -2 one pencil per thread; for the pencil-load kernel 1 one CTA per SM with uncapped registers (two
pencils per thread on 9 warps at 24^3), 2 two CTAs per SM where they fit (16^3), and 3 the
ragged 24^3 form (12 warps, a second pencil for the first 192 threads), 5 one pencil per
thread on 18 warps (24^3, the default there for the owner = target passes; the VJP's u_occ
pass keeps the ragged form).
The pencil-load kernel reads pencil-blocked copies of the orbitals by default; the cases with
HSE_PENCIL_BLOCKS=0 run it on the caller's [x][y][z] arrays.  For every layout the test runs V_x u (owner = target apply), the exchange energy (energy epilogue) and
the full vector-Jacobian product, whose d/d omega term runs the owner = target dot epilogue
(Sec. II C; Eq. "Fock" and its derivative with respect to omega).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_05156_gb300 import hse, inputs

pytestmark = pytest.mark.gpu

LAYOUT_CASES = [(12, -1, 1), (12, -2, 1), (16, -1, 1), (16, -2, 1), (16, 2, 1), (18, -1, 1), (18, -2, 1),
                (20, -1, 1), (20, -2, 1), (8, -1, 1), (8, -2, 1), (24, 1, 1), (24, 3, 1),
                (24, 3, 0), (16, -2, 0), (20, -2, 0), (24, 5, 1), (24, 5, 0)]


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def _rel(got, ref):
    got = np.asarray(got, np.complex128)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("n,variant,blocks", LAYOUT_CASES)
def test_staged_layout_apply_energy_vjp(n, variant, blocks, monkeypatch):
    monkeypatch.setenv("HSE_BLOCKS_PER_SM", str(variant))
    monkeypatch.setenv("HSE_PENCIL_BLOCKS", str(blocks))
    grid = (n, n, n)
    lattice = inputs.cubic_lattice(inputs.A_SI)
    rng = np.random.default_rng(1000 + 10 * n - variant)
    nk, n_occ, n_tgt = 2, 3, 2
    b = 2 * np.pi * np.linalg.inv(lattice).T
    kpts = (rng.random((nk, 3)) - 0.5) @ b
    c64 = lambda x: np.ascontiguousarray(x).astype(np.complex64).astype(np.complex128)
    u_occ = c64(inputs.orthonormal_orbitals(rng, grid, lattice, kpts, n_occ, ecut=60.0))
    u_tgt = c64(inputs.orthonormal_orbitals(rng, grid, lattice, kpts, n_tgt, ecut=60.0))
    ybar = c64(inputs.random_orbitals(int(rng.integers(1 << 30)), u_tgt.shape) * np.abs(u_tgt).mean())
    occ = rng.random((nk, n_occ)) * 0.5 + 0.5
    occ[1, 0] = 0.0  # an empty orbital: skipped partner
    omega, alpha = inputs.OMEGA, inputs.ALPHA
    d = torch.complex64

    plan = hse.Plan(grid, lattice, kpts, n_occ, n_tgt, omega, alpha, dtype=d)
    out = hse.hse_fock_apply(plan, _dev(u_occ, d), _dev(occ, torch.float64), _dev(u_tgt, d))
    hse.hse_status(plan)
    ref = oracle.fock_apply(u_occ, occ, u_tgt, kpts, lattice, grid, omega, alpha)
    assert _rel(out.cpu().numpy(), ref) <= 1e-5

    g_occ, g_tgt, g_om = hse.hse_fock_apply_vjp(plan, _dev(u_occ, d), _dev(occ, torch.float64),
                                                _dev(u_tgt, d), _dev(ybar, d))
    r_occ, r_tgt, r_om = oracle.fock_apply_vjp(u_occ, occ, u_tgt, ybar, kpts, lattice, grid, omega, alpha)
    assert _rel(g_tgt.cpu().numpy(), r_tgt) <= 1e-5
    assert _rel(g_occ.cpu().numpy(), r_occ) <= 1e-5
    assert abs(g_om.item() - r_om) <= 1e-5 * abs(r_om)

    eplan = hse.Plan(grid, lattice, kpts, n_occ, n_occ, omega, alpha, dtype=d)
    e = hse.hse_exchange_energy(eplan, _dev(u_occ, d), _dev(occ, torch.float64)).item()
    e_ref = oracle.exchange_energy(u_occ, occ, kpts, lattice, grid, omega, alpha, 2.0)
    assert e_ref < 0
    assert abs(e - e_ref) <= 1e-5 * abs(e_ref)
