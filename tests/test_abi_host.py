"""C ABI checks that need no GPU: the library builds and loads, exports every symbol the
header declares, and rejects bad problems on the host before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1507_05156_gb300 import _build, hse

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return hse.load_library()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "hse_fock.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hse_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_symbols()
    assert declared, "no declarations parsed"
    assert sorted(hse.EXPORTS) == declared
    for name in declared:
        assert hasattr(lib, name), name


def test_strerror_and_grid_support(lib):
    assert lib.hse_strerror(0) == b"success"
    assert b"overlaps" in lib.hse_strerror(-3)
    for n in (4, 6, 8, 10, 12, 16, 18, 20, 24):
        assert lib.hse_grid_supported(n, hse.HSE_C64) == 1
    assert lib.hse_grid_supported(7, hse.HSE_C64) == 0
    assert lib.hse_grid_supported(7, hse.HSE_C128) == 0
    assert lib.hse_grid_supported(27, hse.HSE_C128) == 1
    assert lib.hse_grid_supported(27, hse.HSE_C64) == 0
    assert lib.hse_grid_supported(15, hse.HSE_C64) == 0  # the fused form needs an even side
    assert lib.hse_grid_supported(15, hse.HSE_C128) == 1
    # the tensor-core option exists for the 24^3 kernel only
    assert lib.hse_grid_supported(24, hse.HSE_C64_TC) == 1
    for n in (8, 16, 20):
        assert lib.hse_grid_supported(n, hse.HSE_C64_TC) == 0
    assert lib.hse_grid_supported(24, 3) == 0  # no such dtype


def _prob(**kw):
    import torch
    args = dict(grid=(8, 8, 8), lattice=np.eye(3) * 10.0, kpts=np.zeros((1, 3)), n_occ=2, n_tgt=2,
                omega=0.106, alpha=0.25, spin_degeneracy=2.0, dtype=torch.complex64)
    args.update(kw)
    return hse._problem(**args)


@pytest.mark.parametrize("kw,code", [
    (dict(grid=(7, 7, 7)), -2),                    # 7 is not a product of 2, 3, 5
    (dict(grid=(8, 8, 12)), -2),                   # fused complex64 form needs a cubic grid
    (dict(grid=(32, 32, 32)), -2),                 # beyond the fused form's 24^3
    (dict(grid=(1, 8, 8)), -1),
    (dict(omega=0.0), -1),
    (dict(omega=float("nan")), -1),
    (dict(n_occ=0), -1),
    (dict(n_tgt=0), -1),
    (dict(lattice=np.zeros((3, 3))), -1),          # singular cell
    (dict(kpts=np.array([[0.0, np.inf, 0.0]])), -1),
    (dict(kpts=np.zeros((2, 3)), kocc=[2]), -1),           # sampled k-point out of range
    (dict(kpts=np.zeros((2, 3)), kocc=[-1]), -1),
    (dict(kpts=np.zeros((2, 3)), kocc=[1, 1]), -1),        # repeated
    (dict(kpts=np.zeros((2, 3)), kocc=[0, 1, 0]), -1),     # more than nk
    (dict(tensor_cores=True), -2),                 # the tensor-core option: 24^3 only
    (dict(grid=(24, 24, 20), tensor_cores=True), -2),
])
def test_plan_create_rejects_bad_problems_on_host(lib, kw, code):
    p, keep = _prob(**kw)
    h = ctypes.c_void_p(123)
    assert lib.hse_plan_create(ctypes.byref(h), ctypes.byref(p)) == code
    assert not h.value


@pytest.mark.parametrize("field,value,code", [
    ("dtype", 3, -1),                  # no such dtype
    ("dtype", -1, -1),
    ("nk", 0, -1),
    ("alpha", float("inf"), -1),
    ("spin_degeneracy", float("nan"), -1),
    ("omega", -0.1, -1),
])
def test_plan_create_rejects_bad_fields_on_host(lib, field, value, code):
    """Fields set on the marshalled struct directly (values the binding would not produce)."""
    p, keep = _prob()
    setattr(p, field, value)
    h = ctypes.c_void_p(123)
    assert lib.hse_plan_create(ctypes.byref(h), ctypes.byref(p)) == code
    assert not h.value


def test_batched_plans_refuse_tensor_core_cells(lib):
    p, keep = _prob(grid=(24, 24, 24), tensor_cores=True)
    cells = (hse.HseProblem * 1)(p)
    h = ctypes.c_void_p(123)
    assert lib.hse_plan_create_batched(ctypes.byref(h), cells, 1) == -2
    assert not h.value


def test_batched_plans_refuse_down_sampling(lib):
    p, keep = _prob(kpts=np.zeros((2, 3)), kocc=[1])
    cells = (hse.HseProblem * 1)(p)
    h = ctypes.c_void_p(123)
    assert lib.hse_plan_create_batched(ctypes.byref(h), cells, 1) == -1
    assert not h.value


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.hse_plan_create(None, None) == -1
    assert lib.hse_plan_create(ctypes.byref(h), None) == -1
    assert lib.hse_fock_apply(None, None, None, None, None, None) == -1
    assert lib.hse_exchange_energy(None, None, None, None, None) == -1
    assert lib.hse_fock_apply_vjp(None, None, None, None, None, None, None, None, None) == -1
    assert lib.hse_status(None, None) == -1
    assert lib.hse_plan_destroy(None) == -1
    assert lib.hse_kinetic_apply(None, None, 1, None, None, None) == -1
    assert lib.hse_taylor_step(None, None, None, None, 0.1, None, None, None) == -1
    assert lib.hse_current(None, None, None, None, None, None) == -1
    assert lib.hse_hartree_potential(None, None, None, None, None) == -1
    assert lib.hse_overlap(None, None, 1, None, None) == -1
    assert lib.hse_orthonormalize(None, None, 1, None) == -1


def test_error_strings(lib):
    for code in range(-8, 0):
        assert lib.hse_strerror(code) != b"unknown error", code
    assert b"linearly dependent" in lib.hse_strerror(-8)
    assert hse.ERRORS[-8] == "HSE_ERR_SINGULAR"
