"""The tensor-core option (HSE_C64_TC): the Y and X axis transforms of every pair convolution
(Sec. II C, Eq. "Fock": pair density -> 3-D FFT -> times the screened kernel -> inverse FFT) as
split-FP16 GEMMs on the tensor cores, against the FP64 oracle at the complex64 tolerance, on
the 24^3 grid the option exists for.  Two k-points (a q = 0 kernel row and a q != 0 one),
owner and partner band counts that leave work items with a single band, and an occupation
pattern with a skipped (f = 0) and a fractional band.  The apply, the exchange energy and the
VJP (the u_tgt pass and the omega-alone dot pass take the tensor-core kernel, the u_occ pass the
FP32 one) are checked; the tensor-core output must also differ from the FP32 kernel's in its
rounding, which shows that the tensor-core kernel ran."""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_05156_gb300 import hse, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5
GRID = (24, 24, 24)


def _dev(x, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def _rel(got, ref):
    return float(np.linalg.norm(np.asarray(got, np.complex128) - ref) / np.linalg.norm(ref))


def _case(seed, nk, n_occ, n_tgt):
    lattice = inputs.cubic_lattice(inputs.A_SI)
    rng = np.random.default_rng(seed)
    b = 2 * np.pi * np.linalg.inv(lattice).T
    kpts = (rng.random((nk, 3)) - 0.5) @ b
    kpts[0] = 0.0
    c64 = lambda x: np.ascontiguousarray(x).astype(np.complex64).astype(np.complex128)
    u_occ = c64(inputs.orthonormal_orbitals(rng, GRID, lattice, kpts, n_occ, ecut=60.0))
    u_tgt = c64(inputs.orthonormal_orbitals(rng, GRID, lattice, kpts, n_tgt, ecut=60.0))
    occ = np.ones((nk, n_occ))
    occ[0, n_occ - 1] = 0.0
    occ[nk - 1, 0] = 0.5
    return lattice, kpts, u_occ, u_tgt, occ


def test_tc_apply_and_energy():
    lattice, kpts, u_occ, u_tgt, occ = _case(2401, 2, 3, 2)
    args = (GRID, lattice, kpts, 3, 2, inputs.OMEGA, inputs.ALPHA)
    got = {}
    for tc in (True, False):
        plan = hse.Plan(*args, tensor_cores=tc)
        got[tc] = hse.hse_fock_apply(plan, _dev(u_occ), _dev(occ, torch.float64), _dev(u_tgt)).cpu().numpy()
        hse.hse_status(plan)
    ref = oracle.fock_apply(u_occ, occ, u_tgt, kpts, lattice, GRID, inputs.OMEGA, inputs.ALPHA)
    err_tc, err_f32 = _rel(got[True], ref), _rel(got[False], ref)
    print(f"24^3 apply, relative error vs FP64: tensor-core {err_tc:.3e}, FP32 {err_f32:.3e}")
    assert err_tc <= TOL
    worst = max(_rel(got[True][k, i], ref[k, i]) for k in range(2) for i in range(2))
    assert worst <= 3 * TOL
    assert not np.array_equal(got[True], got[False])

    eplan = hse.Plan(GRID, lattice, kpts, 3, 3, inputs.OMEGA, inputs.ALPHA, tensor_cores=True)
    e = hse.hse_exchange_energy(eplan, _dev(u_occ), _dev(occ, torch.float64)).item()
    hse.hse_status(eplan)
    e_ref = oracle.exchange_energy(u_occ, occ, kpts, lattice, GRID, inputs.OMEGA, inputs.ALPHA, 2.0)
    print(f"24^3 exchange energy, relative error vs FP64: tensor-core {abs(e - e_ref) / abs(e_ref):.3e}")
    assert e_ref < 0
    assert abs(e - e_ref) <= TOL * abs(e_ref)


def test_tc_vjp():
    lattice, kpts, u_occ, u_tgt, occ = _case(2402, 2, 2, 3)
    ybar = inputs.random_orbitals(2403, u_tgt.shape) * np.abs(u_tgt).mean()
    ybar = ybar.astype(np.complex64).astype(np.complex128)
    plan = hse.Plan(GRID, lattice, kpts, 2, 3, inputs.OMEGA, inputs.ALPHA, tensor_cores=True)
    a = (plan, _dev(u_occ), _dev(occ, torch.float64), _dev(u_tgt), _dev(ybar))
    g_occ, g_tgt, g_om = hse.hse_fock_apply_vjp(*a)
    _, _, g_alone = hse.hse_fock_apply_vjp(*a, need_occ=False, need_tgt=False)
    hse.hse_status(plan)
    r_occ, r_tgt, r_om = oracle.fock_apply_vjp(u_occ, occ, u_tgt, ybar, kpts, lattice, GRID, inputs.OMEGA,
                                               inputs.ALPHA)
    assert _rel(g_tgt.cpu().numpy(), r_tgt) <= TOL
    assert _rel(g_occ.cpu().numpy(), r_occ) <= TOL
    # d/d omega sums terms of both signs: the bound is on the Cauchy-Schwarz scale
    dy = oracle.fock_apply(u_occ, occ, u_tgt, kpts, lattice, GRID, inputs.OMEGA, inputs.ALPHA, kernel="domega")
    scale = np.linalg.norm(ybar) * np.linalg.norm(dy)
    assert abs(g_om.item() - r_om) <= TOL * scale
    assert abs(g_alone.item() - r_om) <= TOL * scale


def test_tc_option_refuses_other_grids_and_dtypes():
    lattice = inputs.cubic_lattice(inputs.A_SI)
    with pytest.raises(RuntimeError):
        hse.Plan((20, 20, 20), lattice, np.zeros((1, 3)), 2, 2, inputs.OMEGA, inputs.ALPHA, tensor_cores=True)
    with pytest.raises(ValueError):
        hse.Plan(GRID, lattice, np.zeros((1, 3)), 2, 2, inputs.OMEGA, inputs.ALPHA, dtype=torch.complex128,
                 tensor_cores=True)


def test_tc_full_24cube_workload_sampled_targets():
    """The timed tensor-core workload (24^3 grid, 8x8x8 k-mesh, 16 occupied + 16 empty targets,
    134,217,728 pair convolutions per apply) in the launch configuration the benchmark times:
    three sampled targets against the oracle element by element, and the exchange energy of
    the tensor-core energy pass against an FP64 dot of the tensor-core apply output."""
    c = inputs.workload(2)
    u_tgt = torch.from_numpy(c.u_tgt.astype(np.complex64)).cuda()
    u_occ = u_tgt[:, :c.n_occ].contiguous()
    occ = torch.from_numpy(c.occ).cuda()
    plan = hse.Plan(c.grid, c.lattice, c.kpts, c.n_occ, c.n_tgt, c.omega, c.alpha, tensor_cores=True)
    out = hse.hse_fock_apply(plan, u_occ, occ, u_tgt)
    hse.hse_status(plan)
    targets = [(0, 0), (261, 15), (511, 31)]
    uo = c.u_occ.astype(np.complex64).astype(np.complex128)
    ut = c.u_tgt.astype(np.complex64).astype(np.complex128)
    ref = oracle.fock_apply(uo, c.occ, ut, c.kpts, c.lattice, c.grid, c.omega, c.alpha, targets=targets)
    got = np.stack([out[k, i].cpu().numpy() for k, i in targets])
    err = _rel(got, ref)
    print(f"24^3 x 8^3 k tensor-core apply, sampled targets: relative error vs FP64 {err:.3e}")
    assert err <= TOL
    plan_e = hse.Plan(c.grid, c.lattice, c.kpts, c.n_occ, c.n_occ, c.omega, c.alpha, tensor_cores=True)
    e = hse.hse_exchange_energy(plan_e, u_occ, occ).item()
    hse.hse_status(plan_e)
    vx = out[:, :c.n_occ].to(torch.complex128)
    dV = abs(np.linalg.det(c.lattice)) / c.npts
    dots = (torch.conj(u_occ.to(torch.complex128)) * vx).real.sum(dim=(2, 3, 4))
    e_ref = 0.5 * 2.0 * dV / c.nk * float((occ * dots).sum())
    assert e < 0
    assert abs(e - e_ref) <= 1e-6 * abs(e_ref)
