"""Batched uneven cells in one persistent, graph-captured launch (hse_fock_apply_batched)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_05156_gb300 import hse, inputs

pytestmark = pytest.mark.gpu


def dev(x, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


def test_small_mixed_batch_vs_oracle_and_graph_replay():
    specs = [((8, 8, 8), (2, 1, 1), 3), ((12, 12, 12), (2, 2, 1), 5), ((16, 16, 16), (1, 1, 2), 3),
             ((8, 8, 8), (1, 1, 1), 9), ((18, 18, 18), (1, 2, 1), 2), ((20, 20, 20), (1, 1, 1), 2),
             ((24, 24, 24), (1, 1, 1), 2)]
    cells = [inputs.make_cell(900 + i, g, km, nb) for i, (g, km, nb) in enumerate(specs)]
    for c in cells:
        c.u_occ = c.u_occ.astype(np.complex64).astype(np.complex128)
        c.u_tgt = c.u_occ
        c.occ = np.random.default_rng(len(c.kpts)).random(c.occ.shape)
    plan = hse.BatchedPlan(cells)
    uo = [dev(c.u_occ) for c in cells]
    oc = [dev(c.occ, torch.float64) for c in cells]
    out1 = hse.hse_fock_apply_batched(plan, uo, oc, uo)          # autotunes, captures the graph
    out2 = hse.hse_fock_apply_batched(plan, uo, oc, uo)          # graph replay
    torch.cuda.synchronize()
    for c, o1, o2 in zip(cells, out1, out2):
        ref = oracle.fock_apply(c.u_occ, c.occ, c.u_occ, c.kpts, c.lattice, c.grid, c.omega, c.alpha)
        assert rel(o1.cpu().numpy(), ref) <= 1e-5
        assert torch.equal(o1, o2)


def test_uneven_batch_32_cells_matches_single_cell_path():
    """32 cells, grids from {12,16,18,20,24}^3, k-meshes 2^3..4^3, 4..16 bands: the batched
    launch against the single-cell launches (same arithmetic, different schedules), and one
    seeded target (k, i) of every cell, 24^3 cells included, element by element against the
    oracle (its full sum over the cell's k' and bands)."""
    cells = inputs.batched_cells()
    assert len(cells) == 32
    plan = hse.BatchedPlan(cells)
    uo = [dev(c.u_occ.astype(np.complex64)) for c in cells]
    oc = [dev(c.occ, torch.float64) for c in cells]
    out = hse.hse_fock_apply_batched(plan, uo, oc, uo)
    torch.cuda.synchronize()
    for c, u, o, x in zip(cells, uo, oc, out):
        p1 = hse.get_plan(c.grid, c.lattice, c.kpts, c.n_occ, c.n_tgt, c.omega, c.alpha, dtype=torch.complex64)
        single = hse.hse_fock_apply(p1, u, o, u)
        assert float((x - single).abs().max() / single.abs().max()) <= 1e-5
    rng = np.random.default_rng(77)
    errs = []
    for i, c in enumerate(cells):
        u64 = c.u_occ.astype(np.complex64).astype(np.complex128)
        targets = [(int(rng.integers(len(c.kpts))), int(rng.integers(c.n_tgt)))]
        ref = oracle.fock_apply(u64, c.occ, u64, c.kpts, c.lattice, c.grid, c.omega, c.alpha, targets=targets)
        got = np.stack([out[i][k, b].cpu().numpy() for k, b in targets])
        errs.append((c.name, rel(got, ref)))
    print("batched cells vs oracle (one target each):", ", ".join(f"{n} {e:.1e}" for n, e in errs))
    assert any(c.grid[0] == 24 for c in cells)
    assert max(e for _, e in errs) <= 1e-5


def test_autotune_cache_round_trip(tmp_path, monkeypatch):
    """HSE_AUTOTUNE_CACHE: the first batched plan times the candidate launch shapes (k' split,
    pencil layouts, serial or concurrent kernels) and stores its choice under a key naming the
    GPU and the cells; a second plan with the same cells reads it back (no timing runs) and
    computes the same result."""
    cache = tmp_path / "autotune.tsv"
    monkeypatch.setenv("HSE_AUTOTUNE_CACHE", str(cache))
    cells = inputs.batched_cells(4)
    uo = [torch.from_numpy(c.u_occ.astype(np.complex64)).cuda() for c in cells]
    oc = [torch.from_numpy(c.occ).cuda() for c in cells]
    first = hse.hse_fock_apply_batched(hse.BatchedPlan(cells), uo, oc, uo)
    torch.cuda.synchronize()
    lines = cache.read_text().splitlines()
    # the stored shape: bits 0-2 the k' split, higher bits the layouts, the serial flag and the
    # per-cell form
    assert len(lines) == 1 and int(lines[0].split("\t")[1]) & 7 in (1, 2, 4)
    second = hse.hse_fock_apply_batched(hse.BatchedPlan(cells), uo, oc, uo)
    torch.cuda.synchronize()
    assert cache.read_text().splitlines() == lines  # served from the cache, nothing appended
    for a, b in zip(first, second):
        assert torch.equal(a, b)


def test_every_tuned_shape_vs_oracle(tmp_path, monkeypatch):
    """The launch shapes the autotuner can choose, forced through the autotune cache: the ragged
    24^3 layout with the kernels one after the other, two pencils a thread on every staged side
    (12^3 then in the 512-thread staged kernel) with a k' split of 2, a split of 4 with the
    defaults (12^3 in its own LayoutOne kernel), and the per-cell form (every cell's single-cell
    launches on parallel branches of the graph); each against the oracle on a batch with every
    supported side."""
    cache = tmp_path / "autotune.tsv"
    monkeypatch.setenv("HSE_AUTOTUNE_CACHE", str(cache))
    specs = [((8, 8, 8), (2, 1, 1), 3), ((12, 12, 12), (2, 2, 1), 3), ((16, 16, 16), (1, 1, 2), 3),
             ((18, 18, 18), (1, 2, 1), 2), ((20, 20, 20), (2, 1, 1), 2), ((24, 24, 24), (2, 1, 1), 2)]
    cells = [inputs.make_cell(950 + i, g, km, nb) for i, (g, km, nb) in enumerate(specs)]
    for c in cells:
        c.u_occ = c.u_occ.astype(np.complex64).astype(np.complex128)
        c.u_tgt = c.u_occ
    uo = [dev(c.u_occ) for c in cells]
    oc = [dev(c.occ, torch.float64) for c in cells]
    refs = [oracle.fock_apply(c.u_occ, c.occ, c.u_occ, c.kpts, c.lattice, c.grid, c.omega, c.alpha) for c in cells]
    hse.hse_fock_apply_batched(hse.BatchedPlan(cells), uo, oc, uo)  # autotunes and stores its line
    torch.cuda.synchronize()
    key = cache.read_text().splitlines()[0].split("\t")[0]
    for shape in (1 | 8 | 16, 2 | 32 | 64 | 128 | 256 | 512, 4, 1 | 1024):
        cache.write_text(f"{key}\t{shape}\n")
        out = hse.hse_fock_apply_batched(hse.BatchedPlan(cells), uo, oc, uo)
        torch.cuda.synchronize()
        for c, o, ref in zip(cells, out, refs):
            assert rel(o.cpu().numpy(), ref) <= 1e-5, (shape, c.grid)


def test_per_cell_form_recaptures_for_new_arrays(tmp_path, monkeypatch):
    """The per-cell form passes the arrays to its kernels as launch arguments, so its graph is
    captured again when a call passes other arrays: calls on two different input copies and
    output buffers, on the first ones again, and once more on the same ones (a replay), each
    against the oracle."""
    cache = tmp_path / "autotune.tsv"
    monkeypatch.setenv("HSE_AUTOTUNE_CACHE", str(cache))
    specs = [((12, 12, 12), (2, 1, 1), 3), ((20, 20, 20), (1, 1, 2), 2), ((24, 24, 24), (2, 1, 1), 2)]
    cells = [inputs.make_cell(970 + i, g, km, nb) for i, (g, km, nb) in enumerate(specs)]
    for c in cells:
        c.u_occ = c.u_occ.astype(np.complex64).astype(np.complex128)
        c.u_tgt = c.u_occ
    refs = [oracle.fock_apply(c.u_occ, c.occ, c.u_occ, c.kpts, c.lattice, c.grid, c.omega, c.alpha) for c in cells]
    uo = [dev(c.u_occ) for c in cells]
    oc = [dev(c.occ, torch.float64) for c in cells]
    hse.hse_fock_apply_batched(hse.BatchedPlan(cells), uo, oc, uo)  # stores the autotune key
    torch.cuda.synchronize()
    key = cache.read_text().splitlines()[0].split("\t")[0]
    cache.write_text(f"{key}\t{1 | 1024}\n")
    plan = hse.BatchedPlan(cells)
    outs = [[torch.full_like(u, float("nan")) for u in uo] for _ in range(2)]
    uo2 = [u.clone() for u in uo]
    for inputs_, out in ((uo, outs[0]), (uo2, outs[1]), (uo, outs[0]), (uo, outs[0])):
        for o in out:
            o.fill_(float("nan"))
        hse.hse_fock_apply_batched(plan, inputs_, oc, inputs_, out=out)
        torch.cuda.synchronize()
        for c, o, ref in zip(cells, out, refs):
            assert rel(o.cpu().numpy(), ref) <= 1e-5, c.grid
