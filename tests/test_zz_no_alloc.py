"""hse_exchange_energy_noalloc: the allocation-free exchange energy.

It serves callers that may not allocate device memory (memory owned by another
allocator, or a loop where cudaMalloc/cudaFree would synchronise the device).  It keeps
its scratch in a static device array instead of a plan.  Checked through the C ABI
against the plan-based hse_exchange_energy and the FP64 oracle, on calls in a row whose
problems differ (so that nothing left in the shared scratch by one call can reach the
next), including a 24^3 problem that runs the pencil-load kernel on the caller's natural
layout.  This file is collected last on purpose, and every test also passes on its own in
a fresh process.
"""
import ctypes
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1507_05156_gb300 import hse, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the complex64 tolerance of the parity tests


def _call_noalloc(lib, prob, u, occ, out):
    return lib.hse_exchange_energy_noalloc(ctypes.byref(prob), ctypes.c_void_p(u.data_ptr()),
                                           ctypes.c_void_p(occ.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


class _Case:
    """One problem: device inputs, the plan-based E_x and the oracle's E_x (FP64, on the
    complex64 values the GPU reads)."""

    def __init__(self, cell, omega, occ_edit=None):
        d = torch.complex64
        self.cell = cell
        occ_np = cell.occ.copy()
        if occ_edit:
            occ_np[occ_edit] = 0.5
        self.u = torch.from_numpy(cell.u_occ.astype(np.complex64)).cuda()
        self.occ = torch.from_numpy(occ_np).cuda()
        plan = hse.get_plan(cell.grid, cell.lattice, cell.kpts, cell.n_occ, cell.n_occ, omega, cell.alpha, dtype=d)
        self.plan_e = hse.hse_exchange_energy(plan, self.u, self.occ).item()
        u64 = cell.u_occ.astype(np.complex64).astype(np.complex128)
        self.oracle_e = oracle.exchange_energy(u64, occ_np, cell.kpts, cell.lattice, cell.grid, omega, cell.alpha, 2.0)
        self.prob, self._keep = hse._problem(cell.grid, cell.lattice, cell.kpts, cell.n_occ, cell.n_occ, omega,
                                             cell.alpha, 2.0, d)

    def check(self, e):
        assert e < 0
        assert abs(e - self.oracle_e) <= TOL * abs(self.oracle_e), (e, self.oracle_e)
        assert abs(e - self.plan_e) <= TOL * abs(self.plan_e), (e, self.plan_e)


def _case_12():
    return _Case(inputs.workload(0), inputs.OMEGA, occ_edit=(3, 1))  # 12^3, 2x2x2 k, 4 bands


def _case_24():
    # 24^3, 2x2x2 k, 4 bands, the paper's omega: its energy pass runs the pencil-load kernel,
    # here on the caller's natural [x][y][z] layout (plans use pencil-blocked copies)
    cell = inputs.make_cell(inputs.SEED_BASE + 207, (24, 24, 24), (2, 2, 2), 4, name="c64_24cube_k2_b4")
    return _Case(cell, inputs.OMEGA_PAPER)


def test_noalloc_energy_matches_plan_and_oracle_on_alternating_problems():
    lib = hse.load_library()
    a, b = _case_12(), _case_24()
    out = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
    free_after_first = None
    for case in (a, b, a, b):
        out.fill_(float("nan"))
        assert _call_noalloc(lib, case.prob, case.u, case.occ, out) == 0
        torch.cuda.synchronize()
        case.check(out.item())
        free = torch.cuda.mem_get_info()[0]
        if free_after_first is None:
            free_after_first = free
        assert free == free_after_first  # no call after the first allocated device memory


def test_noalloc_energy_is_nan_when_a_device_wait_gives_up():
    # the plans' test hook: the staged kernel of the 12^3 energy pass never issues its first
    # partner copy, its bounded wait runs out (no fault), and the energy must not pass for valid
    lib = hse.load_library()
    a = _case_12()
    out = torch.zeros((), dtype=torch.float64, device="cuda")
    os.environ["HSE_INJECT_SKIP_FILL"] = "1"
    try:
        assert _call_noalloc(lib, a.prob, a.u, a.occ, out) == 0
        torch.cuda.synchronize()
    finally:
        del os.environ["HSE_INJECT_SKIP_FILL"]
    assert np.isnan(out.item())
    # the next call starts from a cleared status word and computes correctly
    assert _call_noalloc(lib, a.prob, a.u, a.occ, out) == 0
    torch.cuda.synchronize()
    a.check(out.item())


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = hse.load_library()
    c = inputs.workload(1)  # 20^3 grid with 64 k-points: 4096 kernel rows do not fit
    prob, keep = hse._problem(c.grid, c.lattice, c.kpts, c.n_occ, c.n_occ, c.omega, c.alpha, 2.0, torch.complex64)
    u = torch.empty(16, dtype=torch.complex64, device="cuda")
    occ = torch.empty(1, dtype=torch.float64, device="cuda")
    out = torch.empty((), dtype=torch.float64, device="cuda")
    assert _call_noalloc(lib, prob, u, occ, out) == -1
    # more k-points than the kernel parameters carry (129 > 128), even on a tiny grid
    kp = np.zeros((129, 3))
    prob, keep = hse._problem((4, 4, 4), c.lattice, kp, 1, 1, c.omega, c.alpha, 2.0, torch.complex64)
    assert _call_noalloc(lib, prob, u, occ, out) == -1
