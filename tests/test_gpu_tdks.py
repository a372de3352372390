"""GPU tests of the differentiable exchange operator and the Taylor TDKS harness.

* kinetic term vs the oracle (complex64 fused and complex128 staged);
* torch.autograd.gradcheck of V_x w.r.t. occupied orbitals, targets and omega (complex128);
* a few Taylor steps vs the FP64 oracle propagator;
* the differentiation workload (16^3 grid, 3x3x3 k, 8 bands): 20 fourth-order Taylor steps,
  dt = 0.02, uniform field 0.005 along x, backpropagated with per-step checkpointing; the
  gradient w.r.t. omega and a directional derivative w.r.t. the initial orbitals are checked
  against central finite differences of the same propagation (complex128), and the complex64
  run against the complex128 one within a bound derived from the FP32 rounding per step.
"""
import numpy as np
import pytest
import torch

import oracle
import oracle.tdks as otd
from paper_1507_05156_gb300 import hse, inputs, tdks

pytestmark = pytest.mark.gpu
TRICLINIC = np.array([[7.1, 0.3, -0.4], [0.9, 6.2, 0.5], [-0.6, 1.1, 5.3]])


def dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


def rel(a, b):
    a = np.asarray(a, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dtype,grid,lattice", [(torch.complex64, (12, 12, 12), inputs.cubic_lattice(10.26)),
                                                (torch.complex128, (6, 5, 4), TRICLINIC)])
def test_kinetic_matches_oracle(dtype, grid, lattice):
    rng = np.random.default_rng(1)
    b = 2 * np.pi * np.linalg.inv(lattice).T
    kpts = (rng.random((2, 3)) - 0.5) @ b
    u = inputs.orthonormal_orbitals(rng, grid, lattice, kpts, 3, ecut=60.0)
    if dtype == torch.complex64:
        u = u.astype(np.complex64).astype(np.complex128)
    A = np.array([0.013, -0.004, 0.02])
    plan = hse.get_plan(grid, lattice, kpts, 1, 1, 1.0, 0.25, dtype=dtype)
    got = hse.hse_kinetic_apply(plan, dev(u, dtype), A).cpu().numpy()
    ref = otd.kinetic_apply(u, kpts, lattice, grid, A)
    assert rel(got, ref) <= (1e-5 if dtype == torch.complex64 else 1e-12)


def test_fock_apply_gradcheck_complex128():
    grid = (4, 3, 4)
    rng = np.random.default_rng(2)
    b = 2 * np.pi * np.linalg.inv(TRICLINIC).T
    kpts = (rng.random((2, 3)) - 0.5) @ b
    geom = tdks.Geometry(grid, TRICLINIC, kpts)
    u_occ = dev(inputs.orthonormal_orbitals(rng, grid, TRICLINIC, kpts, 2, ecut=60.0), torch.complex128)
    u_tgt = dev(inputs.orthonormal_orbitals(rng, grid, TRICLINIC, kpts, 2, ecut=60.0), torch.complex128)
    occ = dev(np.array([[1.0, 0.6], [0.8, 1.0]]), torch.float64)
    omega = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    u_occ.requires_grad_(True)
    u_tgt.requires_grad_(True)
    f = lambda a, b_, w: tdks.fock_apply(a, occ, b_, w, geom)
    assert torch.autograd.gradcheck(f, (u_occ, u_tgt, omega), eps=1e-6, atol=1e-8, rtol=1e-5, fast_mode=True)


def _small_tdks_problem(seed, grid=(8, 8, 8), kmesh=(2, 2, 2), nb=4):
    c = inputs.make_cell(seed, grid, kmesh, nb)
    return c


def test_taylor_steps_match_oracle():
    c = _small_tdks_problem(5)
    E = np.array([0.005, 0.0, 0.0])
    ref = otd.propagate(c.u_occ, c.occ, c.kpts, c.lattice, c.grid, c.omega, c.alpha, 0.02, 3, E)
    for dtype, tol in ((torch.complex128, 1e-10), (torch.complex64, 1e-5)):
        geom = tdks.Geometry(c.grid, c.lattice, c.kpts, c.alpha)
        psi0 = dev(c.u_occ.astype(np.complex64) if dtype == torch.complex64 else c.u_occ, dtype)
        occ = dev(c.occ, torch.float64)
        with torch.no_grad():
            got = tdks.propagate(psi0, occ, c.omega, geom, 0.02, 3, E, use_checkpoint=False).cpu().numpy()
        r = ref if dtype == torch.complex128 else otd.propagate(
            c.u_occ.astype(np.complex64).astype(np.complex128), c.occ, c.kpts, c.lattice, c.grid, c.omega, c.alpha,
            0.02, 3, E)
        assert rel(got, r) <= tol


def _loss(psi, w):
    return (torch.conj(w) * psi).real.sum()


def test_differentiation_workload_gradients_vs_finite_differences():
    c = inputs.workload(4)  # 16^3 grid, 3x3x3 k, 8 bands
    E = [0.005, 0.0, 0.0]
    dt, nsteps = 0.02, 20
    geom = tdks.Geometry(c.grid, c.lattice, c.kpts, c.alpha)
    occ = dev(c.occ, torch.float64)
    d = torch.complex128
    psi0 = dev(c.u_occ, d)
    w = dev(inputs.random_orbitals(7, c.u_occ.shape), d)
    direction = dev(inputs.random_orbitals(8, c.u_occ.shape) * np.abs(c.u_occ).mean(), d)

    def run(p0, om, ckpt=True):
        return tdks.propagate(p0, occ, om, geom, dt, nsteps, E, use_checkpoint=ckpt)

    p0 = psi0.clone().requires_grad_(True)
    om = torch.tensor(c.omega, dtype=torch.float64, requires_grad=True)
    L = _loss(run(p0, om), w)
    L.backward()
    g_psi, g_om = p0.grad.clone(), float(om.grad)

    # checkpointed and plain backward agree
    p1 = psi0.clone().requires_grad_(True)
    om1 = torch.tensor(c.omega, dtype=torch.float64, requires_grad=True)
    _loss(run(p1, om1, ckpt=False), w).backward()
    assert torch.allclose(p1.grad, g_psi, rtol=1e-12, atol=1e-14)
    assert abs(float(om1.grad) - g_om) <= 1e-12 * abs(g_om)

    with torch.no_grad():
        h = 1e-6
        fd_om = (float(_loss(run(psi0, c.omega + h), w)) - float(_loss(run(psi0, c.omega - h), w))) / (2 * h)
        e = 1e-5
        fd_dir = (float(_loss(run(psi0 + e * direction, c.omega), w))
                  - float(_loss(run(psi0 - e * direction, c.omega), w))) / (2 * e)
    an_dir = float((torch.conj(g_psi) * direction).real.sum())
    assert abs(g_om - fd_om) <= 1e-6 * abs(fd_om)
    assert abs(an_dir - fd_dir) <= 1e-6 * abs(fd_dir)

    # complex64 run of the same workload against the complex128 one
    p32 = dev(c.u_occ.astype(np.complex64), torch.complex64).requires_grad_(True)
    om32 = torch.tensor(c.omega, dtype=torch.float64, requires_grad=True)
    psi_T32 = run(p32, om32)
    _loss(psi_T32, w.to(torch.complex64)).backward()
    with torch.no_grad():
        psi_T64 = run(psi0, c.omega)
    e_fwd = rel(psi_T32.detach().cpu().numpy(), psi_T64.cpu().numpy())
    e_psi = rel(p32.grad.cpu().numpy(), g_psi.cpu().numpy())
    e_om = abs(float(om32.grad) - g_om) / abs(g_om)
    print(f"complex64 vs complex128 through {nsteps} steps: psi(T) {e_fwd:.2e}, d/dpsi0 {e_psi:.2e}, "
          f"d/domega {e_om:.2e}")
    # Bound (derived, not fitted): each complex64 step rounds the state to FP32 in the four
    # additions of its Taylor terms (4 x 6e-8 = 2.4e-7 relative) and adds the FP32 error of its
    # operator applications scaled by the terms' size (dt |h| about 0.12 on these band-limited
    # orbitals, times about 1.5e-7 per V_x application at 16^3: < 2e-8).  The step maps are
    # close to unitary, so over 20 steps the errors add at most linearly: 20 x 2.6e-7 = 5.2e-6
    # for psi(T).  The backward sweep re-runs the forward and applies the adjoint of every step
    # with the same per-step error, which at most doubles that for the gradients: about 1e-5,
    # the stated complex64 tolerance.
    assert e_fwd <= 5.2e-6
    assert e_psi <= 1e-5
    assert e_om <= 1e-5


# ---------------------------------------------------------------------------
# Fused Taylor step, electric current and the laser-pulse driver vs the FP64 oracle
# ---------------------------------------------------------------------------

def _tdks_cell(seed, grid, lattice, nk, nb, dtype):
    rng = np.random.default_rng(seed)
    b = 2 * np.pi * np.linalg.inv(lattice).T
    kpts = (rng.random((nk, 3)) - 0.5) @ b
    u = inputs.orthonormal_orbitals(rng, grid, lattice, kpts, nb, ecut=60.0)
    if dtype == torch.complex64:
        u = u.astype(np.complex64).astype(np.complex128)
    occ = rng.random((nk, nb)) * 0.5 + 0.5
    return kpts, u, occ


STEP_CASES = [(torch.complex64, (12, 12, 12), inputs.cubic_lattice(10.26), 1e-5),
              (torch.complex128, (6, 5, 4), TRICLINIC, 1e-10)]


@pytest.mark.parametrize("dtype,grid,lattice,tol", STEP_CASES)
def test_fused_taylor_step_matches_oracle(dtype, grid, lattice, tol):
    kpts, u, occ = _tdks_cell(31, grid, lattice, 2, 3, dtype)
    A = np.array([0.011, -0.02, 0.005])
    dt, omega, alpha = 0.05, 0.2, 0.25
    plan = hse.get_plan(grid, lattice, kpts, 3, 3, omega, alpha, dtype=dtype)
    got = hse.hse_taylor_step(plan, dev(u, dtype), dev(occ, torch.float64), A, dt).cpu().numpy()
    ref = otd.taylor_step(u, occ, kpts, lattice, grid, A, omega, alpha, dt)
    # compare the increments psi(t + dt) - psi(t): the step itself, not the carried state
    assert rel(got - u, ref - u) <= tol
    assert rel(got, ref) <= tol


@pytest.mark.parametrize("dtype,grid,lattice,tol", [(torch.complex64, (12, 12, 12), inputs.cubic_lattice(10.26), 1e-12),
                                                    (torch.complex128, (6, 5, 4), TRICLINIC, 1e-12)])
def test_current_matches_oracle(dtype, grid, lattice, tol):
    kpts, u, occ = _tdks_cell(32, grid, lattice, 3, 2, dtype)
    A = np.array([-0.03, 0.012, 0.02])
    plan = hse.get_plan(grid, lattice, kpts, 2, 2, 0.2, 0.25, dtype=dtype)
    J = hse.hse_current(plan, dev(u, dtype), dev(occ, torch.float64), A).cpu().numpy()
    ref = otd.current(u, occ, kpts, lattice, grid, A, 2.0)
    assert np.abs(J - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("dtype,grid,lattice", [(torch.complex64, (12, 12, 12), inputs.cubic_lattice(10.26)),
                                                (torch.complex128, (6, 5, 4), TRICLINIC)])
def test_hartree_potential_matches_oracle(dtype, grid, lattice):
    kpts, u, occ = _tdks_cell(34, grid, lattice, 3, 2, dtype)
    plan = hse.get_plan(grid, lattice, kpts, 2, 2, 0.2, 0.25, dtype=dtype)
    vh = hse.hse_hartree_potential(plan, dev(u, dtype), dev(occ, torch.float64)).cpu().numpy()
    ref = otd.hartree_potential(u, occ, lattice, grid, 2.0)
    assert np.abs(vh - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dtype,grid,lattice,tol", STEP_CASES)
def test_fused_taylor_step_with_hartree_matches_oracle(dtype, grid, lattice, tol):
    kpts, u, occ = _tdks_cell(35, grid, lattice, 2, 3, dtype)
    A = np.array([0.0, 0.01, -0.02])
    dt, omega, alpha = 0.05, 0.2, 0.25
    plan = hse.get_plan(grid, lattice, kpts, 3, 3, omega, alpha, dtype=dtype)
    psi = dev(u, dtype)
    vh = hse.hse_hartree_potential(plan, psi, dev(occ, torch.float64))
    got = hse.hse_taylor_step(plan, psi, dev(occ, torch.float64), A, dt, vloc=vh).cpu().numpy()
    ref = otd.taylor_step(u, occ, kpts, lattice, grid, A, omega, alpha, dt,
                          vloc=otd.hartree_potential(u, occ, lattice, grid, 2.0))
    assert rel(got - u, ref - u) <= tol


@pytest.mark.parametrize("dtype,tol,hartree", [(torch.complex128, 1e-9, False), (torch.complex64, 2e-5, False),
                                               (torch.complex128, 1e-9, True)])
def test_pulse_driver_matches_oracle(dtype, tol, hartree):
    grid, lattice = (8, 8, 8), inputs.cubic_lattice(10.26)
    kpts, u, occ = _tdks_cell(33, grid, lattice, 2, 2, dtype)
    E0, w, Td, d = 0.02, 0.3, 2.0, (0.0, 0.6, 0.8)
    dt, nsteps, omega = 0.1, 12, 0.2
    geom = tdks.Geometry(grid, lattice, kpts, alpha=0.25)
    psi, J, W, drift = tdks.propagate_pulse(dev(u, dtype), dev(occ, torch.float64), omega, geom, dt, nsteps, E0,
                                            w, Td, d, hartree=hartree)
    r_psi, r_J, r_W = otd.propagate_pulse(u, occ, kpts, lattice, grid, omega, 0.25, dt, nsteps, E0, w, Td, d,
                                          hartree=hartree)
    assert rel(psi.cpu().numpy(), r_psi) <= tol
    J = J.cpu().numpy()
    assert np.abs(J - r_J).max() <= tol * np.abs(r_J).max()
    assert np.abs(W - r_W).max() <= tol * np.abs(r_W).max() + 1e-15
    assert np.abs(r_W).max() > 0  # the pulse did work
    # the propagator check: the FP64 overlap drift of the propagated orbitals
    dV = abs(np.linalg.det(lattice)) / np.prod(grid)
    r_S = oracle.ortho.overlap(r_psi, dV)
    r_drift = np.abs(r_S - np.eye(r_S.shape[1])[None]).max()
    assert r_drift > 1e-6  # the 4th-order Taylor step is not unitary
    assert abs(drift - r_drift) <= 20 * tol  # S is off by about twice the orbitals' error
