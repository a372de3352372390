"""d/d omega of the VJP (the derivative of Eq. "Fock", Sec. II C, with respect to the screening
parameter) on both of its GPU paths against the FP64 oracle: computed alone (a pass of its
own) and together with the gradient w.r.t. the occupied orbitals, where it is read off that
pass's transforms by Parseval.  Sizes cover owner tiles with empty slots (8^3: eight owner
slots per CTA, three bands) and the ragged 24^3 kernel.

The cotangent is ybar = u_tgt + 0.3 x noise.  d/d omega = Re <ybar, (d V_x / d omega) u_tgt>:
along u_tgt the operator d V_x / d omega is positive semidefinite (d v / d omega <= 0 and the
-alpha in front), so that part of the sum cannot cancel, and |d/d omega| stays a sizeable
fraction (1.5-10% on these cases) of its Cauchy-Schwarz bound ||ybar|| ||(d V_x/d omega) u_tgt||.
FP32 errors scale with that bound, so the tolerance is taken on it; the test asserts the
fraction is at least 1e-2, which makes the 1e-5 bound a relative check of 1e-3 or better on
the gradient itself.  (A purely random ybar makes the sum cancel to 1e-5 of the bound at 16^3,
where the same tolerance would pin nothing.)"""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_05156_gb300 import hse, inputs

pytestmark = pytest.mark.gpu


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("n,nk,n_occ,n_tgt", [(8, 3, 3, 2), (16, 2, 3, 2), (20, 2, 2, 3), (24, 2, 2, 2)])
def test_omega_gradient_fused_and_alone(n, nk, n_occ, n_tgt):
    grid = (n, n, n)
    lattice = inputs.cubic_lattice(inputs.A_SI)
    rng = np.random.default_rng(300 + n)
    b = 2 * np.pi * np.linalg.inv(lattice).T
    kpts = (rng.random((nk, 3)) - 0.5) @ b
    c64 = lambda x: np.ascontiguousarray(x).astype(np.complex64).astype(np.complex128)
    u_occ = c64(inputs.orthonormal_orbitals(rng, grid, lattice, kpts, n_occ, ecut=60.0))
    u_tgt = c64(inputs.orthonormal_orbitals(rng, grid, lattice, kpts, n_tgt, ecut=60.0))
    noise = inputs.random_orbitals(n, u_tgt.shape) * np.abs(u_tgt).mean()
    ybar = c64(u_tgt + 0.3 * noise)
    occ = rng.random((nk, n_occ)) * 0.5 + 0.5
    d = torch.complex64
    plan = hse.Plan(grid, lattice, kpts, n_occ, n_tgt, inputs.OMEGA, inputs.ALPHA, dtype=d)
    args = (plan, _dev(u_occ, d), _dev(occ, torch.float64), _dev(u_tgt, d), _dev(ybar, d))
    g_occ, _, g_fused = hse.hse_fock_apply_vjp(*args, need_tgt=False)
    _, _, g_alone = hse.hse_fock_apply_vjp(*args, need_occ=False, need_tgt=False)
    hse.hse_status(plan)
    r_occ, _, r_om = oracle.fock_apply_vjp(u_occ, occ, u_tgt, ybar, kpts, lattice, grid, inputs.OMEGA, inputs.ALPHA)
    # FP32 errors scale with the Cauchy-Schwarz bound ||ybar|| ||(d V_x / d omega) u_tgt||
    dy = oracle.fock_apply(u_occ, occ, u_tgt, kpts, lattice, grid, inputs.OMEGA, inputs.ALPHA, kernel="domega")
    scale = np.linalg.norm(ybar) * np.linalg.norm(dy)
    frac = abs(r_om) / scale
    e_fused = abs(g_fused.item() - r_om) / scale
    e_alone = abs(g_alone.item() - r_om) / scale
    print(f"n={n}: |d/domega| / bound = {frac:.3e}; error / bound fused {e_fused:.2e}, alone {e_alone:.2e}; "
          f"relative error fused {e_fused / frac:.2e}, alone {e_alone / frac:.2e}")
    assert 1e-2 <= frac <= 1.0  # the gradient is not a cancelled remainder of its terms
    assert e_fused <= 1e-5
    assert e_alone <= 1e-5
    g_occ = g_occ.cpu().numpy()
    assert np.linalg.norm(g_occ - r_occ) <= 1e-5 * np.linalg.norm(r_occ)
