"""Device-side failure detection without a GPU fault: a bounded wait that nothing satisfies.

A plan created with HSE_INJECT_SKIP_FILL=1 never issues the first partner copy of the staged
complex64 kernel, so the kernel's mbarrier wait runs out (~1 s).  The kernel must record
HSE_ERR_TIMEOUT in the status word, finish without waiting further, and leave the context
usable: a normal plan on the same device afterwards still matches the oracle.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1507_05156_gb300 import hse, inputs

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives(monkeypatch):
    c = inputs.make_cell(77, (12, 12, 12), (1, 1, 1), 4)
    u = torch.from_numpy(c.u_occ.astype(np.complex64)).cuda()
    occ = torch.from_numpy(c.occ).cuda()
    monkeypatch.setenv("HSE_INJECT_SKIP_FILL", "1")
    bad = hse.Plan(c.grid, c.lattice, c.kpts, c.n_occ, c.n_tgt, c.omega, c.alpha)
    monkeypatch.delenv("HSE_INJECT_SKIP_FILL")
    hse.hse_fock_apply(bad, u, occ, u)
    with pytest.raises(hse.HseError) as ei:
        hse.hse_status(bad)
    assert ei.value.code == -5  # HSE_ERR_TIMEOUT
    hse.hse_status(bad)  # the status word was cleared
    good = hse.Plan(c.grid, c.lattice, c.kpts, c.n_occ, c.n_tgt, c.omega, c.alpha)
    out = hse.hse_fock_apply(good, u, occ, u)
    hse.hse_status(good)
    u64 = c.u_occ.astype(np.complex64).astype(np.complex128)
    ref = oracle.fock_apply(u64, c.occ, u64, c.kpts, c.lattice, c.grid, c.omega, c.alpha)
    got = out.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
