"""Out-of-bounds write checks without a sanitizer: every output of the library is placed
between two guard regions filled with a sentinel bit pattern, and the guards must be intact
after the call.  Covers the fused kernels on every path (staged-partner with its running sums
in TMEM and in global memory, the pencil-load kernel with its ragged 24^3 form, the fused
omega gradient), the batched persistent kernels, the FP64 forms, and the Taylor step,
kinetic term, current, Hartree potential, overlap and orthonormalisation."""
import numpy as np
import pytest
import torch

from paper_1507_05156_gb300 import hse, inputs

pytestmark = pytest.mark.gpu

GUARD = 4096  # bytes on each side (a multiple of 16: outputs stay 16-byte aligned)
SENTINEL = 0x5A


class Guarded:
    """A tensor of `shape` and `dtype` inside a byte buffer with sentinel guards."""

    def __init__(self, shape, dtype):
        nbytes = int(np.prod(shape)) * torch.empty((), dtype=dtype).element_size()
        self.buf = torch.full((GUARD + nbytes + GUARD,), SENTINEL, dtype=torch.uint8, device="cuda")
        self.t = self.buf[GUARD:GUARD + nbytes].view(dtype).view(shape)

    def intact(self) -> bool:
        torch.cuda.synchronize()
        return bool((self.buf[:GUARD] == SENTINEL).all() and (self.buf[-GUARD:] == SENTINEL).all())


def _cell(n, nk, n_occ, n_tgt, seed):
    grid = (n, n, n)
    lattice = inputs.cubic_lattice(inputs.A_SI)
    rng = np.random.default_rng(seed)
    b = 2 * np.pi * np.linalg.inv(lattice).T
    kpts = (rng.random((nk, 3)) - 0.5) @ b
    u_occ = inputs.orthonormal_orbitals(rng, grid, lattice, kpts, n_occ, ecut=60.0)
    u_tgt = inputs.orthonormal_orbitals(rng, grid, lattice, kpts, n_tgt, ecut=60.0)
    ybar = inputs.random_orbitals(seed, u_tgt.shape) * np.abs(u_tgt).mean()
    occ = np.ones((nk, n_occ))
    return grid, lattice, kpts, u_occ, u_tgt, ybar, occ


@pytest.mark.parametrize("n,dtype", [(8, torch.complex64), (16, torch.complex64), (20, torch.complex64),
                                     (24, torch.complex64), (12, torch.complex128)])
def test_fock_outputs_stay_in_bounds(n, dtype):
    grid, lattice, kpts, u_occ, u_tgt, ybar, occ = _cell(n, 2, 3, 2, 50 + n)
    dev = lambda x, t=dtype: torch.from_numpy(np.ascontiguousarray(x)).to("cuda", t)
    plan = hse.Plan(grid, lattice, kpts, 3, 2, inputs.OMEGA, inputs.ALPHA, dtype=dtype)
    uo, ut, yb, oc = dev(u_occ), dev(u_tgt), dev(ybar), dev(occ, torch.float64)
    out = Guarded(tuple(u_tgt.shape), dtype)
    hse.hse_fock_apply(plan, uo, oc, ut, out=out.t)
    assert out.intact()
    e = Guarded((), torch.float64)
    eplan = hse.Plan(grid, lattice, kpts, 3, 3, inputs.OMEGA, inputs.ALPHA, dtype=dtype)
    hse.hse_exchange_energy(eplan, uo, oc, out=e.t)
    assert e.intact()
    # the VJP through the library directly, so that every output is guarded
    lib = hse.load_library()
    g_occ, g_tgt, g_om = Guarded(tuple(u_occ.shape), dtype), Guarded(tuple(u_tgt.shape), dtype), \
        Guarded((), torch.float64)
    rc = lib.hse_fock_apply_vjp(plan.handle, hse._ptr(uo), hse._ptr(oc), hse._ptr(ut), hse._ptr(yb),
                                hse._ptr(g_occ.t), hse._ptr(g_tgt.t), hse._ptr(g_om.t), hse._stream())
    assert rc == 0
    hse.hse_status(plan)
    assert g_occ.intact() and g_tgt.intact() and g_om.intact()


def test_batched_outputs_stay_in_bounds():
    cells = inputs.batched_cells(8)
    plan = hse.BatchedPlan(cells)
    uo = [torch.from_numpy(c.u_occ.astype(np.complex64)).cuda() for c in cells]
    oc = [torch.from_numpy(c.occ).cuda() for c in cells]
    outs = [Guarded(tuple(c.u_occ.shape), torch.complex64) for c in cells]
    for _ in range(2):  # the autotuning call and a graph replay
        hse.hse_fock_apply_batched(plan, uo, oc, uo, out=[g.t for g in outs])
    hse.hse_status(plan)
    assert all(g.intact() for g in outs)


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_propagation_and_checks_stay_in_bounds(dtype):
    grid, lattice, kpts, u_occ, _, _, occ = _cell(8, 2, 3, 3, 77)
    dev = lambda x, t=dtype: torch.from_numpy(np.ascontiguousarray(x)).to("cuda", t)
    plan = hse.Plan(grid, lattice, kpts, 3, 3, inputs.OMEGA, inputs.ALPHA, dtype=dtype)
    psi, oc = dev(u_occ), dev(occ, torch.float64)
    A = (0.01, -0.02, 0.03)
    kin = Guarded(tuple(u_occ.shape), dtype)
    hse.hse_kinetic_apply(plan, psi, A, out=kin.t)
    vh = Guarded(grid, torch.float64)
    hse.hse_hartree_potential(plan, psi, oc, out=vh.t)
    step = Guarded(tuple(u_occ.shape), dtype)
    hse.hse_taylor_step(plan, psi, oc, A, 0.05, vloc=vh.t, out=step.t)
    J = Guarded((3,), torch.float64)
    hse.hse_current(plan, psi, oc, A, out=J.t)
    S = Guarded((2, 3, 3), torch.complex128)
    hse.hse_overlap(plan, psi, out=S.t)
    on = Guarded(tuple(u_occ.shape), dtype)
    on.t.copy_(psi)
    hse.hse_orthonormalize(plan, on.t)
    hse.hse_status(plan)
    for g in (kin, vh, step, J, S, on):
        assert g.intact()
