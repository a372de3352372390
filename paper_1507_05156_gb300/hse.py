"""Thin Python binding of the C ABI in include/hse_fock.h (argument marshalling only).

Every step of the Fock-like exchange runs in the CUDA library
``_lib/libhse_fock.so``; this module only checks tensors, passes device pointers and
the current CUDA stream, and keeps plans cached.  If the library is missing or the
tensors are not on a CUDA device it raises: there is no CPU path.

Function names follow the C ABI: hse_fock_apply, hse_exchange_energy,
hse_fock_apply_vjp, hse_fock_apply_batched.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Dict, Optional, Sequence, Tuple

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libhse_fock.so")

HSE_C64 = 0
HSE_C128 = 1
HSE_C64_TC = 2  # complex64, Y/X transforms as split-FP16 tensor-core GEMMs (24^3 grids)

ERRORS = {
    0: "HSE_OK", -1: "HSE_ERR_INVALID_ARG", -2: "HSE_ERR_UNSUPPORTED_GRID", -3: "HSE_ERR_ALIAS",
    -4: "HSE_ERR_CUDA", -5: "HSE_ERR_TIMEOUT", -6: "HSE_ERR_NOMEM", -7: "HSE_ERR_DEVICE",
    -8: "HSE_ERR_SINGULAR",
}

#: every symbol include/hse_fock.h declares
EXPORTS = ("hse_plan_create", "hse_plan_create_batched", "hse_plan_destroy", "hse_fock_apply",
           "hse_exchange_energy", "hse_fock_apply_vjp", "hse_fock_apply_batched", "hse_status",
           "hse_grid_supported", "hse_kernel_launches", "hse_strerror", "hse_exchange_energy_noalloc",
           "hse_kinetic_apply", "hse_taylor_step", "hse_current", "hse_hartree_potential", "hse_overlap",
           "hse_orthonormalize")


class HseError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {ERRORS.get(code, code)}")


class HseProblem(ctypes.Structure):
    _fields_ = [
        ("grid", ctypes.c_int * 3),
        ("lattice", ctypes.c_double * 9),
        ("nk", ctypes.c_int),
        ("kpts", ctypes.POINTER(ctypes.c_double)),
        ("n_occ", ctypes.c_int),
        ("n_tgt", ctypes.c_int),
        ("omega", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("spin_degeneracy", ctypes.c_double),
        ("dtype", ctypes.c_int),
        ("nk_occ", ctypes.c_int),
        ("kocc", ctypes.POINTER(ctypes.c_int)),
    ]


_lib = None
_lib_lock = threading.Lock()


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"HSE CUDA library not built ({path}); run paper_1507_05156_gb300._build.build()")
        lib = ctypes.CDLL(path)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        lib.hse_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(HseProblem)]
        lib.hse_plan_create_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(HseProblem), i]
        lib.hse_plan_destroy.argtypes = [vp]
        lib.hse_fock_apply.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.hse_exchange_energy.argtypes = [vp, vp, vp, vp, vp]
        lib.hse_fock_apply_vjp.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.hse_fock_apply_batched.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.hse_status.argtypes = [vp, vp]
        lib.hse_grid_supported.argtypes = [i, i]
        lib.hse_kernel_launches.argtypes = []
        lib.hse_kernel_launches.restype = ctypes.c_uint64
        lib.hse_exchange_energy_noalloc.argtypes = [ctypes.POINTER(HseProblem), vp, vp, vp, vp]
        lib.hse_exchange_energy_noalloc.restype = i
        lib.hse_kinetic_apply.argtypes = [vp, vp, i, ctypes.POINTER(ctypes.c_double), vp, vp]
        lib.hse_kinetic_apply.restype = i
        lib.hse_taylor_step.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.c_double, vp, vp, vp]
        lib.hse_taylor_step.restype = i
        lib.hse_current.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_double), vp, vp]
        lib.hse_current.restype = i
        lib.hse_hartree_potential.argtypes = [vp, vp, vp, vp, vp]
        lib.hse_hartree_potential.restype = i
        lib.hse_overlap.argtypes = [vp, vp, i, vp, vp]
        lib.hse_overlap.restype = i
        lib.hse_orthonormalize.argtypes = [vp, vp, i, vp]
        lib.hse_orthonormalize.restype = i
        lib.hse_strerror.argtypes = [i]
        lib.hse_strerror.restype = ctypes.c_char_p
        for name in ("hse_plan_create", "hse_plan_create_batched", "hse_plan_destroy", "hse_fock_apply",
                     "hse_exchange_energy", "hse_fock_apply_vjp", "hse_fock_apply_batched", "hse_status",
                     "hse_grid_supported"):
            getattr(lib, name).restype = i
        _lib = lib
        return lib


def _check(code: int, what: str):
    if code != 0:
        raise HseError(code, what)


def kernel_launches() -> int:
    return int(load_library().hse_kernel_launches())


def grid_supported(n: int, dtype: torch.dtype = torch.complex64) -> bool:
    return bool(load_library().hse_grid_supported(int(n), _code(dtype)))


def _code(dtype: torch.dtype) -> int:
    if dtype == torch.complex64:
        return HSE_C64
    if dtype == torch.complex128:
        return HSE_C128
    raise ValueError(f"unsupported dtype {dtype}")


def _problem(grid, lattice, kpts, n_occ, n_tgt, omega, alpha, spin_degeneracy, dtype, kocc=None,
             tensor_cores=False):
    """HseProblem and the host arrays it points to (keep them alive with it)."""
    kp = np.ascontiguousarray(np.asarray(kpts, dtype=np.float64).reshape(-1, 3))
    p = HseProblem()
    p.grid[:] = [int(g) for g in grid]
    p.lattice[:] = [float(x) for x in np.asarray(lattice, dtype=np.float64).reshape(9)]
    p.nk = kp.shape[0]
    p.kpts = kp.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    p.n_occ = int(n_occ)
    p.n_tgt = int(n_tgt)
    p.omega = float(omega)
    p.alpha = float(alpha)
    p.spin_degeneracy = float(spin_degeneracy)
    p.dtype = _code(dtype)
    if tensor_cores:
        if dtype != torch.complex64:
            raise ValueError("tensor_cores needs complex64 orbitals")
        p.dtype = HSE_C64_TC
    if kocc is None:
        p.nk_occ = 0
        ko = None
    else:
        ko = np.ascontiguousarray(np.asarray(kocc, dtype=np.int32).reshape(-1))
        p.nk_occ = int(ko.shape[0])
        p.kocc = ko.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    return p, (kp, ko)


class Plan:
    """An hse_plan: q table, FP64 kernel rows and reduction scratch on one device.

    ``kocc`` (optional) down-samples the Fock sum: the indices of the k-points whose occupied
    orbitals enter it, with weight 1/len(kocc) (Sec. II C, after Eq. "Fock-DS"); the orbital
    arrays keep every k-point.

    ``tensor_cores`` (complex64, 24^3 grids) runs the Y and X axis transforms of the owner =
    target passes as split-FP16 GEMMs on the tensor cores (the library's HSE_C64_TC)."""

    def __init__(self, grid, lattice, kpts, n_occ, n_tgt, omega, alpha, spin_degeneracy=2.0,
                 dtype=torch.complex64, device=None, kocc=None, tensor_cores=False):
        lib = load_library()
        self.grid = tuple(int(g) for g in grid)
        self.nk = int(np.asarray(kpts).reshape(-1, 3).shape[0])
        self.kocc = None if kocc is None else tuple(int(k) for k in kocc)
        self.n_occ, self.n_tgt = int(n_occ), int(n_tgt)
        self.omega, self.alpha, self.spin_degeneracy = float(omega), float(alpha), float(spin_degeneracy)
        self.dtype = dtype
        self.tensor_cores = bool(tensor_cores)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index)
        prob, self._kp = _problem(grid, lattice, kpts, n_occ, n_tgt, omega, alpha, spin_degeneracy, dtype, self.kocc,
                                  self.tensor_cores)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.hse_plan_create(ctypes.byref(h), ctypes.byref(prob)), "hse_plan_create")
        self.handle = h
        self.npts = int(np.prod(self.grid))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.hse_plan_destroy(h)
            self.handle = None

    def shape(self, nbands: int) -> Tuple[int, ...]:
        return (self.nk, nbands) + self.grid


_plan_cache: Dict[tuple, Plan] = {}


def get_plan(grid, lattice, kpts, n_occ, n_tgt, omega, alpha, spin_degeneracy=2.0,
             dtype=torch.complex64, device=None, kocc=None, tensor_cores=False) -> Plan:
    """Plans are cached by every parameter that enters them."""
    dev = torch.cuda.current_device() if device is None else torch.device(device).index
    key = (tuple(int(g) for g in grid), np.asarray(lattice, np.float64).tobytes(),
           np.asarray(kpts, np.float64).tobytes(), int(n_occ), int(n_tgt), float(omega), float(alpha),
           float(spin_degeneracy), dtype, dev, None if kocc is None else tuple(int(k) for k in kocc),
           bool(tensor_cores))
    plan = _plan_cache.get(key)
    if plan is None:
        plan = Plan(grid, lattice, kpts, n_occ, n_tgt, omega, alpha, spin_degeneracy, dtype, device=dev, kocc=kocc,
                    tensor_cores=tensor_cores)
        _plan_cache[key] = plan
    return plan


def _stream(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: Optional[torch.Tensor], plan: Plan, shape, dtype, name: str):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the library has no CPU path)")
    if t.device != plan.device:
        raise ValueError(f"{name} is on {t.device}, plan on {plan.device}")
    if t.dtype != dtype:
        raise ValueError(f"{name} has dtype {t.dtype}, expected {dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _ptr(t: Optional[torch.Tensor]) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def hse_fock_apply(plan: Plan, u_occ: torch.Tensor, occ: torch.Tensor, u_tgt: torch.Tensor,
                   out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """V_x u_tgt for the occupied set (u_occ, occ) on the current stream."""
    lib = load_library()
    _dev(u_occ, plan, plan.shape(plan.n_occ), plan.dtype, "u_occ")
    _dev(u_tgt, plan, plan.shape(plan.n_tgt), plan.dtype, "u_tgt")
    _dev(occ, plan, (plan.nk, plan.n_occ), torch.float64, "occ")
    if out is None:
        out = torch.empty(plan.shape(plan.n_tgt), dtype=plan.dtype, device=plan.device)
    _dev(out, plan, plan.shape(plan.n_tgt), plan.dtype, "out")
    _check(lib.hse_fock_apply(plan.handle, _ptr(u_occ), _ptr(occ), _ptr(u_tgt), _ptr(out), _stream(stream)),
           "hse_fock_apply")
    return out


def hse_exchange_energy(plan: Plan, u_occ: torch.Tensor, occ: torch.Tensor,
                        out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """E_x (FP64, 0-d device tensor) with the targets equal to the occupied set."""
    lib = load_library()
    _dev(u_occ, plan, plan.shape(plan.n_occ), plan.dtype, "u_occ")
    _dev(occ, plan, (plan.nk, plan.n_occ), torch.float64, "occ")
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=plan.device)
    _check(lib.hse_exchange_energy(plan.handle, _ptr(u_occ), _ptr(occ), _ptr(out), _stream(stream)),
           "hse_exchange_energy")
    return out


def hse_fock_apply_vjp(plan: Plan, u_occ, occ, u_tgt, grad_vx, need_occ=True, need_tgt=True, need_omega=True,
                       stream=None):
    """(grad_u_occ, grad_u_tgt, grad_omega); entries not requested are None."""
    lib = load_library()
    _dev(u_occ, plan, plan.shape(plan.n_occ), plan.dtype, "u_occ")
    _dev(u_tgt, plan, plan.shape(plan.n_tgt), plan.dtype, "u_tgt")
    _dev(grad_vx, plan, plan.shape(plan.n_tgt), plan.dtype, "grad_vx")
    _dev(occ, plan, (plan.nk, plan.n_occ), torch.float64, "occ")
    g_occ = torch.empty(plan.shape(plan.n_occ), dtype=plan.dtype, device=plan.device) if need_occ else None
    g_tgt = torch.empty(plan.shape(plan.n_tgt), dtype=plan.dtype, device=plan.device) if need_tgt else None
    g_om = torch.empty((), dtype=torch.float64, device=plan.device) if need_omega else None
    _check(lib.hse_fock_apply_vjp(plan.handle, _ptr(u_occ), _ptr(occ), _ptr(u_tgt), _ptr(grad_vx), _ptr(g_occ),
                                  _ptr(g_tgt), _ptr(g_om), _stream(stream)), "hse_fock_apply_vjp")
    return g_occ, g_tgt, g_om


class BatchedPlan:
    """An hse_plan over many cells (hse_plan_create_batched): one persistent, graph-captured
    launch applies V_x to every cell; the work-item granularity is autotuned on first use."""

    def __init__(self, cells, omega=None, alpha=None, dtype=torch.complex64):
        """cells: objects with grid, lattice, kpts, n_occ, n_tgt, omega, alpha, spin_degeneracy."""
        lib = load_library()
        self.cells = list(cells)
        probs = (HseProblem * len(self.cells))()
        self._keep = []
        for c, cell in enumerate(self.cells):
            pr, kp = _problem(cell.grid, cell.lattice, cell.kpts, cell.n_occ, cell.n_tgt,
                              cell.omega if omega is None else omega, cell.alpha if alpha is None else alpha,
                              getattr(cell, "spin_degeneracy", 2.0), dtype)
            probs[c] = pr
            self._keep.append(kp)
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        _check(lib.hse_plan_create_batched(ctypes.byref(h), probs, len(self.cells)), "hse_plan_create_batched")
        self.handle = h
        self.dtype = dtype

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.hse_plan_destroy(h)
            self.handle = None


def hse_fock_apply_batched(plan: BatchedPlan, u_occ, occ, u_tgt, out=None, stream=None):
    """V_x for every cell of a batched plan; lists of per-cell device tensors."""
    lib = load_library()
    n = len(plan.cells)
    if not (len(u_occ) == len(occ) == len(u_tgt) == n):
        raise ValueError("one tensor per cell is required")
    if out is None:
        out = [torch.empty_like(t) for t in u_tgt]
    for c, cell in enumerate(plan.cells):
        nk = len(cell.kpts)
        for name, t, shape, dt in (("u_occ", u_occ[c], (nk, cell.n_occ) + tuple(cell.grid), plan.dtype),
                                   ("u_tgt", u_tgt[c], (nk, cell.n_tgt) + tuple(cell.grid), plan.dtype),
                                   ("out", out[c], (nk, cell.n_tgt) + tuple(cell.grid), plan.dtype),
                                   ("occ", occ[c], (nk, cell.n_occ), torch.float64)):
            if not t.is_cuda or t.dtype != dt or tuple(t.shape) != shape or not t.is_contiguous():
                raise ValueError(f"cell {c}: {name} must be a contiguous CUDA {dt} tensor of shape {shape}")
    arr = lambda ts: (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
    _check(lib.hse_fock_apply_batched(plan.handle, arr(u_occ), arr(occ), arr(u_tgt), arr(out), _stream(stream)),
           "hse_fock_apply_batched")
    return out


def hse_kinetic_apply(plan: Plan, u: torch.Tensor, A, out: Optional[torch.Tensor] = None,
                      stream=None) -> torch.Tensor:
    """1/2 |G + k + A|^2 applied to the orbitals u [nk][nbands][grid] (the plan's dtype)."""
    lib = load_library()
    if u.dim() != 5 or u.shape[0] != plan.nk or tuple(u.shape[2:]) != plan.grid:
        raise ValueError(f"u has shape {tuple(u.shape)}, expected ({plan.nk}, nbands) + {plan.grid}")
    nb = int(u.shape[1])
    _dev(u, plan, plan.shape(nb), plan.dtype, "u")
    if out is None:
        out = torch.empty_like(u)
    _dev(out, plan, plan.shape(nb), plan.dtype, "out")
    a = (ctypes.c_double * 3)(*[float(x) for x in np.asarray(A, dtype=np.float64).reshape(3)])
    _check(lib.hse_kinetic_apply(plan.handle, _ptr(u), nb, a, _ptr(out), _stream(stream)), "hse_kinetic_apply")
    return out


def _vec3(A):
    return (ctypes.c_double * 3)(*[float(x) for x in np.asarray(A, dtype=np.float64).reshape(3)])


def hse_taylor_step(plan: Plan, psi: torch.Tensor, occ: torch.Tensor, A, dt: float,
                    vloc: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
                    stream=None) -> torch.Tensor:
    """One fourth-order Taylor step psi -> sum_n (-i dt h)^n / n! psi, h = T[A] + v_loc + V_x[psi]
    frozen over the step (the plan's occupied set is psi; n_tgt == n_occ); vloc: float64 grid."""
    lib = load_library()
    _dev(psi, plan, plan.shape(plan.n_occ), plan.dtype, "psi")
    _dev(occ, plan, (plan.nk, plan.n_occ), torch.float64, "occ")
    _dev(vloc, plan, plan.grid, torch.float64, "vloc")
    if out is None:
        out = torch.empty_like(psi)
    _dev(out, plan, plan.shape(plan.n_occ), plan.dtype, "out")
    _check(lib.hse_taylor_step(plan.handle, _ptr(psi), _ptr(occ), _vec3(A), float(dt), _ptr(vloc), _ptr(out),
                               _stream(stream)), "hse_taylor_step")
    return out


def hse_hartree_potential(plan: Plan, psi: torch.Tensor, occ: torch.Tensor, out: Optional[torch.Tensor] = None,
                          stream=None) -> torch.Tensor:
    """Hartree potential (float64 grid on the device) of the density of psi [nk][n_occ][grid]."""
    lib = load_library()
    _dev(psi, plan, plan.shape(plan.n_occ), plan.dtype, "psi")
    _dev(occ, plan, (plan.nk, plan.n_occ), torch.float64, "occ")
    if out is None:
        out = torch.empty(plan.grid, dtype=torch.float64, device=plan.device)
    _dev(out, plan, plan.grid, torch.float64, "out")
    _check(lib.hse_hartree_potential(plan.handle, _ptr(psi), _ptr(occ), _ptr(out), _stream(stream)),
           "hse_hartree_potential")
    return out


def hse_current(plan: Plan, psi: torch.Tensor, occ: torch.Tensor, A, out: Optional[torch.Tensor] = None,
                stream=None) -> torch.Tensor:
    """Electric current J (device float64 [3]) of the orbitals psi [nk][n_occ][grid]."""
    lib = load_library()
    _dev(psi, plan, plan.shape(plan.n_occ), plan.dtype, "psi")
    _dev(occ, plan, (plan.nk, plan.n_occ), torch.float64, "occ")
    if out is None:
        out = torch.empty(3, dtype=torch.float64, device=plan.device)
    _dev(out, plan, (3,), torch.float64, "out")
    _check(lib.hse_current(plan.handle, _ptr(psi), _ptr(occ), _vec3(A), _ptr(out), _stream(stream)), "hse_current")
    return out


def _bands(plan: Plan, u: torch.Tensor) -> int:
    if u.dim() != 5 or u.shape[0] != plan.nk or tuple(u.shape[2:]) != plan.grid:
        raise ValueError(f"u has shape {tuple(u.shape)}, expected ({plan.nk}, nbands) + {plan.grid}")
    nb = int(u.shape[1])
    _dev(u, plan, plan.shape(nb), plan.dtype, "u")
    return nb


def hse_overlap(plan: Plan, u: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """FP64 overlap matrices S[k][a][b] = dV sum_r conj(u_a) u_b (complex128 [nk][nb][nb])."""
    lib = load_library()
    nb = _bands(plan, u)
    if out is None:
        out = torch.empty((plan.nk, nb, nb), dtype=torch.complex128, device=plan.device)
    _dev(out, plan, (plan.nk, nb, nb), torch.complex128, "out")
    _check(lib.hse_overlap(plan.handle, _ptr(u), nb, _ptr(out), _stream(stream)), "hse_overlap")
    return out


def hse_orthonormalize(plan: Plan, u: torch.Tensor, stream=None) -> torch.Tensor:
    """Orthonormalises u [nk][nb][grid] in place per k-point (FP64 modified Gram-Schmidt, twice);
    a linearly dependent band surfaces as HSE_ERR_SINGULAR from hse_status."""
    lib = load_library()
    nb = _bands(plan, u)
    _check(lib.hse_orthonormalize(plan.handle, _ptr(u), nb, _stream(stream)), "hse_orthonormalize")
    return u


def hse_status(plan: Plan, stream=None) -> None:
    _check(load_library().hse_status(plan.handle, _stream(stream)), "hse_status")
