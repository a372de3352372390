"""hse_exchange_energy_noalloc: the allocation-free exchange energy.

It serves callers that may not allocate device memory (memory owned by another
allocator, or a loop where cudaMalloc/cudaFree would synchronise the device).  It keeps
its scratch in a static device array instead of a plan.  Checked through the C ABI
against the plan-based hse_exchange_energy on two calls in a row.  This file is collected
last on purpose, and the test also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1507_05156_gb300 import hse, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the complex64 tolerance of the parity tests


def _call_noalloc(lib, prob, u, occ, out):
    return lib.hse_exchange_energy_noalloc(ctypes.byref(prob), ctypes.c_void_p(u.data_ptr()),
                                           ctypes.c_void_p(occ.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_energy_matches_plan_energy_twice():
    lib = hse.load_library()
    c = inputs.workload(0)  # 12^3 grid, 2x2x2 k, 4 bands
    d = torch.complex64
    u = torch.from_numpy(c.u_occ.astype(np.complex64)).cuda()
    occ_np = c.occ.copy()
    occ_np[3, 1] = 0.5
    occ = torch.from_numpy(occ_np).cuda()
    plan = hse.get_plan(c.grid, c.lattice, c.kpts, c.n_occ, c.n_occ, c.omega, c.alpha, dtype=d)
    ref = hse.hse_exchange_energy(plan, u, occ).item()
    assert ref < 0

    prob, keep = hse._problem(c.grid, c.lattice, c.kpts, c.n_occ, c.n_occ, c.omega, c.alpha, 2.0, d)
    out = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        assert _call_noalloc(lib, prob, u, occ, out) == 0
        torch.cuda.synchronize()
        e = out.item()
        assert abs(e - ref) <= TOL * abs(ref), (e, ref)


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = hse.load_library()
    c = inputs.workload(1)  # 20^3 grid with 64 k-points: 4096 kernel rows do not fit
    prob, keep = hse._problem(c.grid, c.lattice, c.kpts, c.n_occ, c.n_occ, c.omega, c.alpha, 2.0, torch.complex64)
    u = torch.empty(16, dtype=torch.complex64, device="cuda")
    occ = torch.empty(1, dtype=torch.float64, device="cuda")
    out = torch.empty((), dtype=torch.float64, device="cuda")
    assert _call_noalloc(lib, prob, u, occ, out) == -1
