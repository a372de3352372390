"""GPU parity of the CUDA library against the FP64 oracle (element by element).

Tolerances (relative L2 over the whole output, plus the worst single target):
  complex64 fused form  1e-5   (FP32 pair convolutions, FP64 reductions)
  complex128 staged     1e-10
The oracle always runs on the exact values the GPU received (complex64 inputs are
widened to complex128 before the oracle sees them), so the error is the kernel's own.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_05156_gb300 import hse, inputs

pytestmark = pytest.mark.gpu

TOL = {torch.complex64: 1e-5, torch.complex128: 1e-10}
TRICLINIC = np.array([[7.1, 0.3, -0.4], [0.9, 6.2, 0.5], [-0.6, 1.1, 5.3]])


def rel_err(got, ref):
    got = np.asarray(got, np.complex128)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def worst_target(got, ref):
    g = np.asarray(got, np.complex128).reshape(ref.shape[0] * ref.shape[1], -1)
    r = ref.reshape(g.shape)
    return float(max(np.linalg.norm(a - b) / np.linalg.norm(b) for a, b in zip(g, r)))


def to_dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def rounded(x, dtype):
    return x.astype(np.complex64).astype(np.complex128) if dtype == torch.complex64 else x


def small_cell(seed, grid, nk, n_occ, n_tgt, lattice=None, occ_pattern=False):
    lattice = inputs.cubic_lattice(inputs.A_SI) if lattice is None else lattice
    rng = np.random.default_rng(seed)
    b = 2 * np.pi * np.linalg.inv(lattice).T
    kpts = (rng.random((nk, 3)) - 0.5) @ b
    u = inputs.orthonormal_orbitals(rng, grid, lattice, kpts, max(n_occ, n_tgt), ecut=60.0)
    u_occ = np.ascontiguousarray(u[:, :n_occ])
    u_tgt = np.ascontiguousarray(inputs.orthonormal_orbitals(rng, grid, lattice, kpts, n_tgt, ecut=60.0))
    occ = np.ones((nk, n_occ))
    if occ_pattern:
        occ = rng.random((nk, n_occ))
        occ[0, 0] = 0.0  # a skipped (empty) orbital
    return lattice, kpts, u_occ, occ, u_tgt


def run_apply(lattice, kpts, u_occ, occ, u_tgt, grid, omega, alpha, dtype):
    plan = hse.get_plan(grid, lattice, kpts, u_occ.shape[1], u_tgt.shape[1], omega, alpha, dtype=dtype)
    out = hse.hse_fock_apply(plan, to_dev(u_occ, dtype), to_dev(occ, torch.float64), to_dev(u_tgt, dtype))
    hse.hse_status(plan)
    return out.cpu().numpy()


# (grid side, nk, n_occ, n_tgt): tails chosen so that n_tgt is not a multiple of the
# CTA's owner slots (4^3: 32, 6^3: 16, 8^3: 8, 10^3/12^3: 4, 16^3: 2)
CUBIC_CASES = [(4, 2, 3, 33), (6, 2, 2, 17), (8, 3, 3, 9), (10, 2, 2, 5), (12, 2, 3, 5),
               (16, 2, 2, 3), (18, 2, 2, 2), (20, 2, 2, 2), (24, 2, 2, 2)]


@pytest.mark.parametrize("n,nk,n_occ,n_tgt", CUBIC_CASES)
@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_apply_cubic_grids(n, nk, n_occ, n_tgt, dtype):
    grid = (n, n, n)
    lattice, kpts, u_occ, occ, u_tgt = small_cell(100 + n, grid, nk, n_occ, n_tgt, occ_pattern=True)
    u_occ, u_tgt = rounded(u_occ, dtype), rounded(u_tgt, dtype)
    got = run_apply(lattice, kpts, u_occ, occ, u_tgt, grid, 0.106, 0.25, dtype)
    ref = oracle.fock_apply(u_occ, occ, u_tgt, kpts, lattice, grid, 0.106, 0.25)
    assert rel_err(got, ref) <= TOL[dtype]
    assert worst_target(got, ref) <= 3 * TOL[dtype]


@pytest.mark.parametrize("grid", [(6, 5, 4), (12, 10, 9), (2, 3, 5)])
def test_apply_noncubic_triclinic_fp64(grid):
    lattice, kpts, u_occ, occ, u_tgt = small_cell(7, grid, 3, 2, 3, lattice=TRICLINIC, occ_pattern=True)
    got = run_apply(lattice, kpts, u_occ, occ, u_tgt, grid, 0.3, 0.25, torch.complex128)
    ref = oracle.fock_apply(u_occ, occ, u_tgt, kpts, lattice, grid, 0.3, 0.25)
    assert rel_err(got, ref) <= 1e-10


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_apply_triclinic_cubic_grid(dtype):
    grid = (8, 8, 8)
    lattice, kpts, u_occ, occ, u_tgt = small_cell(8, grid, 3, 3, 4, lattice=TRICLINIC)
    u_occ, u_tgt = rounded(u_occ, dtype), rounded(u_tgt, dtype)
    got = run_apply(lattice, kpts, u_occ, occ, u_tgt, grid, inputs.OMEGA_PAPER, 0.25, dtype)
    ref = oracle.fock_apply(u_occ, occ, u_tgt, kpts, lattice, grid, inputs.OMEGA_PAPER, 0.25)
    assert rel_err(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_workload_fp64_12cube_full(dtype):
    c = inputs.workload(0)
    u = rounded(c.u_occ, dtype)
    got = run_apply(c.lattice, c.kpts, u, c.occ, u, c.grid, c.omega, c.alpha, dtype)
    ref = oracle.fock_apply(u, c.occ, u, c.kpts, c.lattice, c.grid, c.omega, c.alpha)
    assert rel_err(got, ref) <= TOL[dtype]
    assert worst_target(got, ref) <= 3 * TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_exchange_energy(dtype):
    c = inputs.workload(0)
    u = rounded(c.u_occ, dtype)
    occ = c.occ.copy()
    occ[1, 2] = 0.5
    plan = hse.get_plan(c.grid, c.lattice, c.kpts, c.n_occ, c.n_occ, c.omega, c.alpha, dtype=dtype)
    e = hse.hse_exchange_energy(plan, to_dev(u, dtype), to_dev(occ, torch.float64)).item()
    ref = oracle.exchange_energy(u, occ, c.kpts, c.lattice, c.grid, c.omega, c.alpha, 2.0)
    assert ref < 0
    assert abs(e - ref) <= TOL[dtype] * abs(ref)


def test_vjp_complex64():
    grid = (8, 8, 8)
    lattice, kpts, u_occ, occ, u_tgt = small_cell(21, grid, 3, 3, 5, lattice=TRICLINIC, occ_pattern=True)
    u_occ, u_tgt = rounded(u_occ, torch.complex64), rounded(u_tgt, torch.complex64)
    ybar = rounded(inputs.random_orbitals(22, u_tgt.shape) * np.abs(u_tgt).mean(), torch.complex64)
    omega, alpha = 0.2, 0.25
    plan = hse.get_plan(grid, lattice, kpts, 3, 5, omega, alpha, dtype=torch.complex64)
    d = torch.complex64
    g_occ, g_tgt, g_om = hse.hse_fock_apply_vjp(plan, to_dev(u_occ, d), to_dev(occ, torch.float64),
                                                to_dev(u_tgt, d), to_dev(ybar, d))
    r_occ, r_tgt, r_om = oracle.fock_apply_vjp(u_occ, occ, u_tgt, ybar, kpts, lattice, grid, omega, alpha)
    assert rel_err(g_tgt.cpu().numpy(), r_tgt) <= 1e-5
    assert rel_err(g_occ.cpu().numpy(), r_occ) <= 1e-5
    assert abs(g_om.item() - r_om) <= 1e-5 * abs(r_om)


@pytest.mark.parametrize("grid,nk", [((6, 5, 4), 3), ((8, 8, 8), 1)])
def test_vjp_complex128(grid, nk):
    lattice, kpts, u_occ, occ, u_tgt = small_cell(23, grid, nk, 3, 4, lattice=TRICLINIC, occ_pattern=True)
    ybar = inputs.random_orbitals(24, u_tgt.shape) * np.abs(u_tgt).mean()
    omega, alpha = 0.2, 0.25
    d = torch.complex128
    plan = hse.get_plan(grid, lattice, kpts, 3, 4, omega, alpha, dtype=d)
    g_occ, g_tgt, g_om = hse.hse_fock_apply_vjp(plan, to_dev(u_occ, d), to_dev(occ, torch.float64),
                                                to_dev(u_tgt, d), to_dev(ybar, d))
    r_occ, r_tgt, r_om = oracle.fock_apply_vjp(u_occ, occ, u_tgt, ybar, kpts, lattice, grid, omega, alpha)
    assert rel_err(g_tgt.cpu().numpy(), r_tgt) <= 1e-10
    assert rel_err(g_occ.cpu().numpy(), r_occ) <= 1e-10
    assert abs(g_om.item() - r_om) <= 1e-10 * abs(r_om)


def test_deterministic_and_f_zero_skips():
    grid = (12, 12, 12)
    lattice, kpts, u_occ, occ, u_tgt = small_cell(31, grid, 2, 3, 5, occ_pattern=True)
    a = run_apply(lattice, kpts, u_occ, occ, u_tgt, grid, 0.106, 0.25, torch.complex64)
    b = run_apply(lattice, kpts, u_occ, occ, u_tgt, grid, 0.106, 0.25, torch.complex64)
    assert np.array_equal(a, b)
    occ0 = np.zeros_like(occ)
    z = run_apply(lattice, kpts, u_occ, occ0, u_tgt, grid, 0.106, 0.25, torch.complex64)
    assert not np.any(z)


def test_alias_and_shape_errors():
    grid = (8, 8, 8)
    lattice, kpts, u_occ, occ, u_tgt = small_cell(41, grid, 2, 2, 2)
    d = torch.complex64
    plan = hse.get_plan(grid, lattice, kpts, 2, 2, 0.106, 0.25, dtype=d)
    uo, ut = to_dev(u_occ, d), to_dev(u_tgt, d)
    oc = to_dev(occ, torch.float64)
    with pytest.raises(hse.HseError) as ei:
        hse.hse_fock_apply(plan, uo, oc, ut, out=ut)
    assert ei.value.code == -3
    with pytest.raises(ValueError):
        hse.hse_fock_apply(plan, uo.cpu(), oc, ut)


def test_bench_workload_sampled_targets():
    """The 20^3, 4x4x4 k, 16-band workload at full size, in the launch configuration the
    bench times; six sampled targets are checked element by element against the oracle."""
    c = inputs.workload(1)
    u = rounded(c.u_occ, torch.complex64)
    got = run_apply(c.lattice, c.kpts, u, c.occ, u, c.grid, c.omega, c.alpha, torch.complex64)
    rng = np.random.default_rng(5)
    targets = [(int(rng.integers(c.nk)), int(rng.integers(c.n_tgt))) for _ in range(6)]
    ref = oracle.fock_apply(u, c.occ, u, c.kpts, c.lattice, c.grid, c.omega, c.alpha, targets=targets)
    g = np.stack([got[k, i] for k, i in targets])
    assert rel_err(g, ref) <= 1e-5


def test_many_partners_beyond_occupation_cache():
    """One k-point with 1100 occupied bands: a work item then has more partners than the
    staged kernel caches in shared memory (1024), exercising its global-memory path; the
    orbitals need not be orthonormal for the operator."""
    grid = (4, 4, 4)
    lattice = inputs.cubic_lattice(inputs.A_SI)
    kpts = np.array([[0.03, -0.02, 0.01]])
    u_occ = rounded(inputs.random_orbitals(51, (1, 1100) + grid) * 0.06, torch.complex64)
    u_tgt = rounded(inputs.random_orbitals(52, (1, 3) + grid) * 0.06, torch.complex64)
    occ = np.random.default_rng(53).random((1, 1100))
    occ[0, ::7] = 0.0
    got = run_apply(lattice, kpts, u_occ, occ, u_tgt, grid, 0.106, 0.25, torch.complex64)
    ref = oracle.fock_apply(u_occ, occ, u_tgt, kpts, lattice, grid, 0.106, 0.25)
    assert rel_err(got, ref) <= 1e-5


def test_workload_24cube_k8_sampled_and_energy_consistency():
    """24^3 grid, 8x8x8 k-mesh (512 k), 16 occupied + 16 empty targets: 134,217,728 pair
    convolutions in one apply.  Three sampled targets (occupied and empty bands) are checked
    element by element against the oracle, and so are their expectation values
    dV <u_i|V_x u_i>; the FP64 exchange-energy reduction is checked against an FP64 dot of the
    full complex64 output computed on the host."""
    c = inputs.workload(2)
    d = torch.complex64
    u_tgt = torch.from_numpy(c.u_tgt.astype(np.complex64)).cuda()
    u_occ = u_tgt[:, :c.n_occ].contiguous()
    occ = torch.from_numpy(c.occ).cuda()
    plan = hse.get_plan(c.grid, c.lattice, c.kpts, c.n_occ, c.n_tgt, c.omega, c.alpha, dtype=d)
    out = hse.hse_fock_apply(plan, u_occ, occ, u_tgt)
    hse.hse_status(plan)
    targets = [(137, 5), (402, 23), (9, 0)]
    uo = c.u_occ.astype(np.complex64).astype(np.complex128)
    ut = c.u_tgt.astype(np.complex64).astype(np.complex128)
    ref = oracle.fock_apply(uo, c.occ, ut, c.kpts, c.lattice, c.grid, c.omega, c.alpha, targets=targets)
    got = np.stack([out[k, i].cpu().numpy() for k, i in targets])
    assert rel_err(got, ref) <= 1e-5
    # per-target expectation values dV <u_i | V_x u_i> (the terms of E_x, Sec. V Eq. "Eex01"):
    # the oracle's against the GPU output's, both reduced in FP64 on the host
    dV = abs(np.linalg.det(c.lattice)) / c.npts
    for t, (k, i) in enumerate(targets):
        e_ref = dV * np.real(np.vdot(ut[k, i], ref[t]))
        e_gpu = dV * np.real(np.vdot(ut[k, i], got[t].astype(np.complex128)))
        assert e_ref < 0
        assert abs(e_gpu - e_ref) <= 1e-6 * abs(e_ref), (k, i, e_gpu, e_ref)
    # E_x from the fused energy epilogue vs an FP64 dot of the apply output (occupied block)
    plan_e = hse.get_plan(c.grid, c.lattice, c.kpts, c.n_occ, c.n_occ, c.omega, c.alpha, dtype=d)
    e = hse.hse_exchange_energy(plan_e, u_occ, occ).item()
    vx = out[:, :c.n_occ].to(torch.complex128)
    dV = abs(np.linalg.det(c.lattice)) / c.npts
    dots = (torch.conj(u_occ.to(torch.complex128)) * vx).real.sum(dim=(2, 3, 4))
    e_ref = 0.5 * 2.0 * dV / c.nk * float((occ * dots).sum())
    assert e < 0
    assert abs(e - e_ref) <= 1e-6 * abs(e_ref)
