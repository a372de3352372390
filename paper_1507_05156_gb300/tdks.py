"""Differentiable Fock-like exchange and a Taylor-series TDKS propagator on the GPU.

* ``FockApply`` is the autograd form of hse_fock_apply: forward runs the fused (complex64) or
  staged (complex128) kernels, backward runs hse_fock_apply_vjp for the gradients with
  respect to the occupied orbitals, the target orbitals and omega.  Passing the same tensor
  as occupied and target set (the self-consistent case) gives the summed gradient.
* ``KineticApply`` applies 1/2 |G + k + A|^2 (hse_kinetic_apply); the operator is Hermitian,
  so its vector-Jacobian product is the same operator applied to the cotangent.
* ``taylor_step`` / ``propagate`` follow Sec. II C of arXiv:1507.05156: psi(t + dt) =
  sum_{n<=4} (-i dt h)^n / n! psi(t), with h = T[A(t)] + V_x[psi(t)] frozen over the step.
  ``propagate`` recomputes each step in the backward pass (activation checkpointing), so
  only one set of orbitals per step is kept.
* ``propagate_pulse`` drives the orbitals with the sin^2 pulse of Sec. IV,
  A(t) = -(E0 / w) cos(w t) sin^2(pi t / T_d), through the library's fused Taylor step
  (hse_taylor_step, no autograd) and records the current J(t) (hse_current, Sec. II A without
  the nonlocal part) and the energy absorbed per unit volume W(t) = int J . E dt (Sec. V).
* ``overlap_drift``: max |S - 1| of the FP64 overlap matrices of a set of orbitals
  (hse_overlap), the check of a propagation (the Taylor step is not unitary).

Every operator application runs in the CUDA library; PyTorch only holds the tensors, forms
the Taylor sum and drives autograd.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np
import torch
from torch.utils.checkpoint import checkpoint

from . import hse


class Geometry:
    """Cell, k-points and HSE parameters shared by every call of one problem.  ``kocc``
    optionally down-samples the Fock sum to those k-point indices (weight 1/len(kocc))."""

    def __init__(self, grid, lattice, kpts, alpha=0.25, spin_degeneracy=2.0, kocc=None):
        self.grid = tuple(int(g) for g in grid)
        self.lattice = np.asarray(lattice, dtype=np.float64)
        self.kpts = np.asarray(kpts, dtype=np.float64).reshape(-1, 3)
        self.alpha = float(alpha)
        self.spin_degeneracy = float(spin_degeneracy)
        self.kocc = None if kocc is None else tuple(int(k) for k in kocc)

    def plan(self, n_occ, n_tgt, omega, dtype):
        return hse.get_plan(self.grid, self.lattice, self.kpts, n_occ, n_tgt, float(omega), self.alpha,
                            self.spin_degeneracy, dtype=dtype, kocc=self.kocc)


class FockApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u_occ, u_tgt, omega, occ, geom: Geometry):
        plan = geom.plan(u_occ.shape[1], u_tgt.shape[1], float(omega), u_occ.dtype)
        out = hse.hse_fock_apply(plan, u_occ.contiguous(), occ, u_tgt.contiguous())
        ctx.save_for_backward(u_occ, u_tgt, occ)
        ctx.plan = plan
        ctx.omega_dtype, ctx.omega_device = omega.dtype, omega.device
        return out

    @staticmethod
    def backward(ctx, grad_out):
        u_occ, u_tgt, occ = ctx.saved_tensors
        g_occ, g_tgt, g_om = hse.hse_fock_apply_vjp(
            ctx.plan, u_occ.contiguous(), occ, u_tgt.contiguous(), grad_out.contiguous(),
            need_occ=ctx.needs_input_grad[0], need_tgt=ctx.needs_input_grad[1], need_omega=ctx.needs_input_grad[2])
        if g_om is not None:
            g_om = g_om.to(device=ctx.omega_device, dtype=ctx.omega_dtype)
        return g_occ, g_tgt, g_om, None, None


class KineticApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, A, geom: Geometry):
        plan = geom.plan(1, 1, 1.0, u.dtype)  # the kinetic term does not use omega or bands
        ctx.plan, ctx.A = plan, A
        return hse.hse_kinetic_apply(plan, u.contiguous(), A)

    @staticmethod
    def backward(ctx, grad_out):
        return hse.hse_kinetic_apply(ctx.plan, grad_out.contiguous(), ctx.A), None, None


def fock_apply(u_occ, occ, u_tgt, omega, geom: Geometry):
    if not torch.is_tensor(omega):
        omega = torch.tensor(float(omega), dtype=torch.float64)
    return FockApply.apply(u_occ, u_tgt, omega, occ, geom)


def kinetic_apply(u, A, geom: Geometry):
    return KineticApply.apply(u, tuple(float(a) for a in A), geom)


def hamiltonian_apply(psi_frozen, occ, phi, omega, A, geom: Geometry):
    """h phi = T[A] phi + V_x[psi_frozen] phi."""
    return kinetic_apply(phi, A, geom) + fock_apply(psi_frozen, occ, phi, omega, geom)


def taylor_step(psi, occ, omega, A, dt, geom: Geometry, order: int = 4):
    """sum_{n=0}^{order} (-i dt h)^n / n! psi, h frozen at psi (Sec. II C)."""
    out = psi
    term = psi
    for n in range(1, order + 1):
        term = (-1j * dt / n) * hamiltonian_apply(psi, occ, term, omega, A, geom)
        out = out + term
    return out


def propagate(psi0, occ, omega, geom: Geometry, dt: float, nsteps: int, efield: Sequence[float],
              use_checkpoint: bool = True):
    """nsteps Taylor steps with A(t_s) = -efield t_s, t_s = s dt (field switched on at t = 0)."""
    E = np.asarray(efield, dtype=np.float64)
    psi = psi0
    for s in range(nsteps):
        A = tuple(float(a) for a in (-E * (s * dt)))
        if use_checkpoint:
            psi = checkpoint(taylor_step, psi, occ, omega, A, dt, geom, use_reentrant=False)
        else:
            psi = taylor_step(psi, occ, omega, A, dt, geom)
    return psi


def pulse_vector_potential(t: float, E0: float, w: float, Td: float, direction) -> np.ndarray:
    """A(t) = -(E0 / w) cos(w t) sin^2(pi t / T_d) along ``direction`` inside (0, T_d), else 0."""
    if not 0.0 < t < Td:
        return np.zeros(3)
    return -(E0 / w) * np.cos(w * t) * np.sin(np.pi * t / Td) ** 2 * np.asarray(direction, dtype=np.float64)


def pulse_field(t: float, E0: float, w: float, Td: float, direction) -> np.ndarray:
    """E(t) = -dA/dt of pulse_vector_potential."""
    if not 0.0 < t < Td:
        return np.zeros(3)
    ph, env = w * t, np.pi * t / Td
    dA_dt = (E0 / w) * (w * np.sin(ph) * np.sin(env) ** 2 - np.cos(ph) * (np.pi / Td) * np.sin(2.0 * env))
    return -dA_dt * np.asarray(direction, dtype=np.float64)


def overlap_drift(plan: hse.Plan, psi: torch.Tensor) -> float:
    """max over k, a, b of |S_ab - delta_ab|, S = dV sum_r conj(psi_a) psi_b in FP64 on the GPU."""
    S = hse.hse_overlap(plan, psi)
    eye = torch.eye(S.shape[1], dtype=S.dtype, device=S.device)
    return float((S - eye).abs().max().item())


def propagate_pulse(psi0: torch.Tensor, occ: torch.Tensor, omega: float, geom: Geometry, dt: float, nsteps: int,
                    E0: float, w: float, Td: float, direction, hartree: bool = False):
    """nsteps fused Taylor steps under the pulse.  Step s (t_s = s dt) uses h frozen at psi(t_s)
    with A(t_s) (and, with ``hartree``, the Hartree potential of psi(t_s)); J_s = J(t_s) from
    psi(t_s) and A(t_s); W by the trapezoidal rule on J . E.
    Returns (psi(t_nsteps), J [nsteps+1][3] float64 on the device, W [nsteps+1] numpy, the
    overlap drift max |S - 1| of psi(t_nsteps))."""
    plan = geom.plan(psi0.shape[1], psi0.shape[1], omega, psi0.dtype)
    bufs = [psi0.contiguous().clone(), torch.empty_like(psi0)]
    J = torch.empty((nsteps + 1, 3), dtype=torch.float64, device=psi0.device)
    for s in range(nsteps + 1):
        A = pulse_vector_potential(s * dt, E0, w, Td, direction)
        hse.hse_current(plan, bufs[0], occ, A, out=J[s])
        if s < nsteps:
            vh = hse.hse_hartree_potential(plan, bufs[0], occ) if hartree else None
            hse.hse_taylor_step(plan, bufs[0], occ, A, dt, vloc=vh, out=bufs[1])
            bufs.reverse()
    Jh = J.cpu().numpy()
    E = np.stack([pulse_field(s * dt, E0, w, Td, direction) for s in range(nsteps + 1)])
    p = np.einsum("sc,sc->s", Jh, E)
    W = np.concatenate([[0.0], np.cumsum(0.5 * dt * (p[1:] + p[:-1]))])
    return bufs[0], J, W, overlap_drift(plan, bufs[0])
