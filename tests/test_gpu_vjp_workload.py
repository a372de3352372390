"""The vector-Jacobian product on the differentiation workload (16^3 grid, 3x3x3 Monkhorst-Pack
k-mesh, 8 bands; 46,656 ordered pairs per apply) against the FP64 oracle's gradient, element by
element, in both precisions: hse_fock_apply_vjp's gradients w.r.t. u_occ, u_tgt and omega
against oracle.fock_apply_vjp (the adjoint of Eq. "Fock-DS", Sec. II C, written out in the
paper's order).

Inputs are complex64-representable (rounded once), so one oracle evaluation serves both
precisions.  Occupations vary (0.5 .. 1).  The cotangent is ybar = u + 0.3 x noise, so that the
omega gradient is not a cancelled remainder of its terms (see test_gpu_vjp_omega.py); it is
checked on its Cauchy-Schwarz scale ||ybar|| ||(d V_x / d omega) u||.  Tolerances: relative L2
over each gradient array 1e-5 (complex64) / 1e-10 (complex128), and the worst single orbital
within 3x that.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_05156_gb300 import hse, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload_and_oracle():
    c = inputs.workload(4)
    u = c.u_occ.astype(np.complex64).astype(np.complex128)
    occ = 0.5 + 0.5 * np.random.default_rng(44).random(c.occ.shape)
    noise = inputs.random_orbitals(41, u.shape) * np.abs(u).mean()
    ybar = (u + 0.3 * noise).astype(np.complex64).astype(np.complex128)
    r_occ, r_tgt, r_om = oracle.fock_apply_vjp(u, occ, u, ybar, c.kpts, c.lattice, c.grid, c.omega, c.alpha)
    dy = oracle.fock_apply(u, occ, u, c.kpts, c.lattice, c.grid, c.omega, c.alpha, kernel="domega")
    scale = np.linalg.norm(ybar) * np.linalg.norm(dy)
    return c, u, occ, ybar, (r_occ, r_tgt, r_om), scale


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _worst_orbital(a, b):
    d = np.linalg.norm((a - b).reshape(a.shape[0] * a.shape[1], -1), axis=1)
    r = np.linalg.norm(b.reshape(b.shape[0] * b.shape[1], -1), axis=1)
    return float(np.max(d / r))


@pytest.mark.parametrize("dtype,tol", [(torch.complex64, 1e-5), (torch.complex128, 1e-10)])
def test_vjp_differentiation_workload_vs_oracle(workload_and_oracle, dtype, tol):
    c, u, occ, ybar, (r_occ, r_tgt, r_om), scale = workload_and_oracle
    plan = hse.get_plan(c.grid, c.lattice, c.kpts, c.n_occ, c.n_tgt, c.omega, c.alpha, dtype=dtype)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)
    ud = dev(u)
    g_occ, g_tgt, g_om = hse.hse_fock_apply_vjp(plan, ud, torch.from_numpy(occ).cuda(), ud, dev(ybar))
    hse.hse_status(plan)
    g_occ = g_occ.cpu().numpy().astype(np.complex128)
    g_tgt = g_tgt.cpu().numpy().astype(np.complex128)
    frac = abs(r_om) / scale
    errs = {"u_occ": _rel(g_occ, r_occ), "u_tgt": _rel(g_tgt, r_tgt),
            "u_occ worst orbital": _worst_orbital(g_occ, r_occ), "u_tgt worst orbital": _worst_orbital(g_tgt, r_tgt),
            "omega / bound": abs(g_om.item() - r_om) / scale}
    print(f"{dtype}: |d/domega| / bound = {frac:.3e};", ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    assert frac >= 1e-2
    assert errs["u_occ"] <= tol and errs["u_tgt"] <= tol
    assert errs["u_occ worst orbital"] <= 3 * tol and errs["u_tgt worst orbital"] <= 3 * tol
    assert errs["omega / bound"] <= tol
