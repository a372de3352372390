"""Out-of-memory handling of plans, simulated on the host (no real exhaustion of the GPU).

The test hook HSE_FAIL_ALLOC_AT=k, read when a plan is created, makes the plan's k-th device
allocation (0-based, over the plan's life) fail as cudaMalloc does when the device is out of
memory, without allocating.  Every failure must come back as HSE_ERR_NOMEM, free what was
allocated before it (free device memory does not shrink when the same failure is repeated),
and a plan whose allocation on first use failed must stay usable.
"""
import numpy as np
import pytest
import torch

from paper_1507_05156_gb300 import hse, inputs

pytestmark = pytest.mark.gpu

NOMEM = -6


def _free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _creation_failures(make, monkeypatch):
    """Fail each allocation of a plan's creation in turn; returns how many there are."""
    for k in range(200):
        monkeypatch.setenv("HSE_FAIL_ALLOC_AT", str(k))
        frees = []
        for _ in range(3):
            try:
                plan = make()
            except hse.HseError as e:
                assert e.code == NOMEM, (k, e)
                frees.append(_free())
                continue
            del plan
            monkeypatch.delenv("HSE_FAIL_ALLOC_AT")
            return k
        assert frees[2] == frees[1] == frees[0], (k, frees)  # nothing left behind
    raise AssertionError("plan creation never succeeded")


@pytest.mark.parametrize("dtype,kocc", [(torch.complex64, None), (torch.complex128, None), (torch.complex64, [0, 3])])
def test_plan_creation_out_of_memory(dtype, kocc, monkeypatch):
    c = inputs.make_cell(inputs.SEED_BASE + 310, (12, 12, 12), (2, 2, 1), 3)
    make = lambda: hse.Plan(c.grid, c.lattice, c.kpts, c.n_occ, c.n_tgt, c.omega, c.alpha, dtype=dtype, kocc=kocc)
    n = _creation_failures(make, monkeypatch)
    assert n >= 8  # q table, k-points, kernel rows (FP64 and FP32, value and d/d omega), partials, status


def test_batched_plan_creation_out_of_memory(monkeypatch):
    cells = inputs.batched_cells(3)
    n = _creation_failures(lambda: hse.BatchedPlan(cells), monkeypatch)
    assert n >= 8


def test_allocation_on_first_use_fails_then_recovers(monkeypatch):
    # a 24^3 apply copies its orbitals into pencil-blocked plan scratch allocated on first use
    c = inputs.make_cell(inputs.SEED_BASE + 311, (24, 24, 24), (1, 1, 1), 2)
    make = lambda: hse.Plan(c.grid, c.lattice, c.kpts, c.n_occ, c.n_tgt, c.omega, c.alpha)
    n_create = _creation_failures(make, monkeypatch)
    u = torch.from_numpy(c.u_occ.astype(np.complex64)).cuda()
    occ = torch.from_numpy(c.occ).cuda()
    plan0 = make()
    ref = hse.hse_fock_apply(plan0, u, occ, u)
    hse.hse_status(plan0)
    monkeypatch.setenv("HSE_FAIL_ALLOC_AT", str(n_create))  # the first allocation after creation
    plan = make()
    monkeypatch.delenv("HSE_FAIL_ALLOC_AT")
    with pytest.raises(hse.HseError) as err:
        hse.hse_fock_apply(plan, u, occ, u)
    assert err.value.code == NOMEM
    out = hse.hse_fock_apply(plan, u, occ, u)  # the next call allocates and computes
    hse.hse_status(plan)
    assert torch.equal(out, ref)
