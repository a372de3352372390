"""The oracle's pins catch plausible mistakes (no GPU needed).

Each case plants one mistake in a copy of an oracle module's source, on the CPU: a dropped
term, a wrong sign, a wrong index, a transposed operand or a wrong normalisation in one step
of Sec. II C (kernel, pair density, transforms, q = k - k', the k' sum and its weights, E_x,
the VJP), of the time step and its diagnostics (kinetic term, Taylor series, current, pulse,
Hartree potential) or of the overlap / Gram-Schmidt checks.  The mutated copy replaces the
module's functions for the duration of the case, and at least one of the listed pins of
``test_oracle_pins.py``, ``test_oracle_tdks.py`` or ``test_oracle_ortho.py`` must then fail.
The pins compare the oracle with closed forms, explicit O(N^2) sums, invariants, a matrix
exponential and finite differences, never with itself, so every mutant below is caught by
something outside the oracle.
"""
import inspect
import types

import pytest

import oracle
import oracle.ortho
import oracle.tdks
from oracle import hse_oracle

import test_oracle_ortho as PO
import test_oracle_pins as P
import test_oracle_tdks as PT

# the planted mistakes may divide by zero or overflow on their way to a failing pin
pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

# (name, snippet of the oracle's source, its mutated form, pins that must catch it)
MUTANTS = [
    ("kernel unscreened (bare Coulomb 4 pi / g^2)",
     "out[~small] = -np.expm1(-xs) / xs", "out[~small] = 1.0 / xs",
     [lambda: P.test_screened_kernel_closed_form(0.106), P.test_plane_wave_closed_form_including_pi_over_omega2_limit]),
    ("kernel limit at g = 0 dropped",
     "out[small] = 1.0", "out[small] = 0.0",
     [lambda: P.test_screened_kernel_closed_form(0.106), P.test_plane_wave_closed_form_including_pi_over_omega2_limit]),
    ("kernel exponent g^2 / 2 omega^2",
     "x = g2 / (4.0 * omega * omega)", "x = g2 / (2.0 * omega * omega)",
     [lambda: P.test_screened_kernel_closed_form(0.106), P.test_screened_kernel_small_g_series]),
    ("d v / d omega with the wrong sign",
     "return -(2.0 * np.pi / omega ** 3)", "return (2.0 * np.pi / omega ** 3)",
     [P.test_screened_kernel_omega_derivative, P.test_vjp_matches_central_finite_differences]),
    ("pair density without the conjugate",
     "return np.conj(u_j) * u_i", "return u_j * u_i",
     [P.test_plane_wave_closed_form_including_pi_over_omega2_limit, P.test_fft_form_equals_realspace_double_sum]),
    ("pair density conjugating the wrong factor",
     "return np.conj(u_j) * u_i", "return u_j * np.conj(u_i)",
     [P.test_plane_wave_closed_form_including_pi_over_omega2_limit, P.test_fft_form_equals_realspace_double_sum]),
    ("q = k' - k",
     "q = kpts[k] - kpts[kp]\n            v = kernel_on_grid(grid, lattice, q, omega, derivative=(kernel == \"domega\"))",
     "q = kpts[kp] - kpts[k]\n            v = kernel_on_grid(grid, lattice, q, omega, derivative=(kernel == \"domega\"))",
     [P.test_plane_wave_closed_form_including_pi_over_omega2_limit,
      P.test_supercell_at_gamma_equals_primitive_cell_with_two_kpoints]),
    ("forward transform without 1/N",
     "return sfft.fftn(rho, axes=(-3, -2, -1), norm=\"forward\", workers=_workers())",
     "return sfft.fftn(rho, axes=(-3, -2, -1), norm=\"backward\", workers=_workers())",
     [lambda: P.test_forward_transform_equals_direct_sum((4, 4, 4)),
      P.test_plane_wave_closed_form_including_pi_over_omega2_limit]),
    ("inverse transform with the forward exponent",
     "return sfft.ifftn(rt, axes=(-3, -2, -1), norm=\"forward\", workers=_workers())",
     "return sfft.fftn(rt, axes=(-3, -2, -1), norm=\"backward\", workers=_workers())",
     [lambda: P.test_forward_transform_equals_direct_sum((4, 4, 4)),
      P.test_plane_wave_closed_form_including_pi_over_omega2_limit]),
    ("reciprocal basis transposed",
     "return 2.0 * np.pi * np.linalg.inv(A).T", "return 2.0 * np.pi * np.linalg.inv(A)",
     [P.test_g_vectors_are_dual_to_grid_positions, P.test_plane_wave_closed_form_including_pi_over_omega2_limit]),
    ("Nyquist index +N/2 instead of -N/2",
     "return np.where(idx <= (n - 1) // 2, idx, idx - n)", "return np.where(idx <= n // 2, idx, idx - n)",
     [P.test_integer_frequencies_match_fftfreq_convention]),
    ("accumulation with conj(u_j)",
     "acc += np.einsum(\"j,j...,jt...->t...\", occ[kp], u_j, phi)",
     "acc += np.einsum(\"j,j...,jt...->t...\", occ[kp], np.conj(u_j), phi)",
     [P.test_plane_wave_closed_form_including_pi_over_omega2_limit, P.test_fft_form_equals_realspace_double_sum]),
    ("occupation of the target k-point instead of k'",
     "acc += np.einsum(\"j,j...,jt...->t...\", occ[kp], u_j, phi)",
     "acc += np.einsum(\"j,j...,jt...->t...\", occ[k], u_j, phi)",
     [P.test_fft_form_equals_realspace_double_sum, P.test_plane_wave_closed_form_including_pi_over_omega2_limit]),
    ("1/N_k weight dropped",
     "out[rows] = -alpha / len(kps) * acc", "out[rows] = -alpha * acc",
     [P.test_plane_wave_closed_form_including_pi_over_omega2_limit, P.test_constant_kernel_limit_is_a_local_product]),
    ("down-sampled sum weighted 1/N_k instead of 1/N_q",
     "out[rows] = -alpha / len(kps) * acc", "out[rows] = -alpha / nk * acc",
     [P.test_downsampled_plane_wave_closed_form]),
    ("down-sampled VJP weighted 1/N_k instead of 1/N_q",
     "c = alpha * occ[kp] / len(kps)", "c = alpha * occ[kp] / nk",
     [P.test_downsampled_hermitian_negative_and_vjp_by_finite_differences]),
    ("exchange with the wrong sign",
     "out[rows] = -alpha / len(kps) * acc", "out[rows] = alpha / len(kps) * acc",
     [P.test_hermitian_and_negative_semidefinite, P.test_plane_wave_closed_form_including_pi_over_omega2_limit]),
    ("E_x without the 1/2",
     "return 0.5 * spin_degeneracy * e / nk", "return spin_degeneracy * e / nk",
     [P.test_exchange_energy_negative_and_gradient_by_finite_difference]),
    ("E_x without the occupation weight",
     "e += occ[k][i] * dV * np.real(np.vdot(u_occ[k, i], vx[k, i]))",
     "e += dV * np.real(np.vdot(u_occ[k, i], vx[k, i]))",
     [P.test_exchange_energy_negative_and_gradient_by_finite_difference]),
    ("E_x from |<u, V_x u>| instead of the real part",
     "e += occ[k][i] * dV * np.real(np.vdot(u_occ[k, i], vx[k, i]))",
     "e += occ[k][i] * dV * np.abs(np.vdot(u_occ[k, i], vx[k, i]))",
     [P.test_exchange_energy_negative_and_gradient_by_finite_difference]),
    ("VJP w.r.t. u_occ missing its second term",
     "np.conj(phi) * y_i[None, :] + u_i[None, :] * np.conj(psib))",
     "np.conj(phi) * y_i[None, :])",
     [P.test_vjp_matches_central_finite_differences]),
    ("VJP w.r.t. u_tgt through phi instead of psibar",
     "g_tgt[k] += -np.einsum(\"j,j...,jt...->t...\", c, u_j, psib)",
     "g_tgt[k] += -np.einsum(\"j,j...,jt...->t...\", c, u_j, phi)",
     [P.test_vjp_matches_central_finite_differences]),
    ("VJP w.r.t. omega with the wrong sign",
     "g_omega += float(np.real(np.vdot(y_i, dy)))", "g_omega -= float(np.real(np.vdot(y_i, dy)))",
     [P.test_vjp_matches_central_finite_differences]),
    ("brute-force real-space sum without 1/N",
     "M = K[diff[..., 0], diff[..., 1], diff[..., 2]] / N",
     "M = K[diff[..., 0], diff[..., 1], diff[..., 2]]",
     [P.test_fft_form_equals_realspace_double_sum]),
    ("direct DFT with the inverse exponent",
     "ph = np.exp(-2j * np.pi", "ph = np.exp(2j * np.pi",
     [lambda: P.test_forward_transform_equals_direct_sum((4, 4, 4))]),
]


TDKS_MUTANTS = [
    ("kinetic term without the 1/2",
     "fac = 0.5 * np.sum(gk * gk, axis=-1)", "fac = np.sum(gk * gk, axis=-1)",
     [PT.test_kinetic_on_plane_wave_closed_form]),
    ("kinetic term with A subtracted",
     "gk = G + np.asarray(kpts[k]) + np.asarray(A, dtype=np.float64)\n        fac",
     "gk = G + np.asarray(kpts[k]) - np.asarray(A, dtype=np.float64)\n        fac",
     [PT.test_kinetic_on_plane_wave_closed_form]),
    ("Taylor series with +i dt",
     "term = (-1j * dt / n) * hamiltonian_apply(", "term = (1j * dt / n) * hamiltonian_apply(",
     [PT.test_taylor_step_matches_matrix_exponential_to_fifth_order]),
    ("Taylor series without the 1/n!",
     "term = (-1j * dt / n) * hamiltonian_apply(", "term = (-1j * dt) * hamiltonian_apply(",
     [PT.test_taylor_step_matches_matrix_exponential_to_fifth_order, PT.test_taylor_norm_drift_closed_form]),
    ("Taylor series stopping at third order",
     "for n in range(1, order + 1):\n        term = (-1j", "for n in range(1, order):\n        term = (-1j",
     [PT.test_taylor_norm_drift_closed_form, PT.test_taylor_step_matches_matrix_exponential_to_fifth_order]),
    ("local potential dropped from h",
     "out = out + np.asarray(vloc, dtype=np.float64).reshape(grid) * np.asarray(phi).reshape(out.shape)",
     "out = out + 0.0 * np.asarray(vloc, dtype=np.float64).reshape(grid)",
     [PT.test_hamiltonian_on_plane_wave_with_local_potential_closed_form]),
    ("propagation with A(t) = +E t",
     "psi = taylor_step(psi, occ, kpts, lattice, grid, -E * (s * dt), omega, alpha, dt)",
     "psi = taylor_step(psi, occ, kpts, lattice, grid, E * (s * dt), omega, alpha, dt)",
     [PT.test_propagate_uses_vector_potential_of_time]),
    ("current with the wrong sign",
     "J -= spin_degeneracy / nk * np.einsum(", "J += spin_degeneracy / nk * np.einsum(",
     [PT.test_current_of_plane_waves_closed_form, PT.test_current_diamagnetic_shift_and_zero_for_real_orbitals]),
    ("current without A (no diamagnetic term)",
     "gk = G + np.asarray(kpts[k]) + np.asarray(A, dtype=np.float64)       # [grid][3]",
     "gk = G + np.asarray(kpts[k])       # [grid][3]",
     [PT.test_current_diamagnetic_shift_and_zero_for_real_orbitals]),
    ("pulse field with the wrong sign",
     "return -dA * d", "return dA * d",
     [PT.test_pulse_field_is_minus_dA_dt_and_vanishes_outside]),
    ("work by the rectangle rule on the new current only",
     "Ws.append(Ws[-1] + 0.5 * dt * (Js[-2] @ e0 + Js[-1] @ e1))", "Ws.append(Ws[-1] + dt * (Js[-1] @ e1))",
     [PT.test_pulse_on_free_plane_wave_work_closed_form]),
    ("Hartree kernel 4 pi / |G| instead of 4 pi / |G|^2",
     "fac[nz] = 4.0 * np.pi / g2[nz]", "fac[nz] = 4.0 * np.pi / np.sqrt(g2[nz])",
     [PT.test_hartree_of_two_plane_waves_closed_form]),
    ("Hartree potential keeping G = 0 (no neutralising background)",
     "nz = g2 > 0", "nz = g2 >= 0",
     [PT.test_hartree_of_uniform_density_vanishes_and_energy_is_nonnegative]),
    ("density without the spin degeneracy",
     "return spin_degeneracy / u.shape[0] * np.einsum(", "return 1.0 / u.shape[0] * np.einsum(",
     [PT.test_hartree_of_uniform_density_vanishes_and_energy_is_nonnegative,
      PT.test_hartree_of_two_plane_waves_closed_form]),
    ("Hartree energy without the 1/2",
     "return float(0.5 * dV * np.sum(vh * rho))", "return float(dV * np.sum(vh * rho))",
     [PT.test_hartree_of_two_plane_waves_closed_form]),
]

ORTHO_MUTANTS = [
    ("overlap without dV",
     "return dV * np.einsum(\"kar,kbr->kab\", np.conj(v), v)", "return np.einsum(\"kar,kbr->kab\", np.conj(v), v)",
     [PO.test_overlap_of_plane_waves_closed_form]),
    ("overlap conjugating the ket",
     "return dV * np.einsum(\"kar,kbr->kab\", np.conj(v), v)", "return dV * np.einsum(\"kar,kbr->kab\", v, np.conj(v))",
     [PO.test_overlap_of_plane_waves_closed_form]),
    ("Gram-Schmidt projection with the bra and ket swapped",
     "v[k, a] -= (dV * np.vdot(v[k, b], v[k, a])) * v[k, b]", "v[k, a] -= (dV * np.vdot(v[k, a], v[k, b])) * v[k, b]",
     [PO.test_gram_schmidt_equals_qr_with_positive_diagonal,
      PO.test_gram_schmidt_of_orthonormal_set_is_identity_and_result_is_orthonormal]),
    ("Gram-Schmidt without the normalisation",
     "v[k, a] /= np.sqrt(dV * np.vdot(v[k, a], v[k, a]).real)", "v[k, a] /= 1.0",
     [PO.test_gram_schmidt_equals_qr_with_positive_diagonal]),
]


def _load(module: types.ModuleType, old: str, new: str) -> types.ModuleType:
    """A copy of `module` with `old` (present exactly once) replaced by `new`."""
    src = inspect.getsource(module)
    assert src.count(old) == 1, f"snippet not found exactly once: {old!r}"
    mod = types.ModuleType(module.__name__ + "_mutant")
    mod.__file__ = module.__file__
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new), module.__file__ + " (mutant)", "exec"), mod.__dict__)
    return mod


def _install(monkeypatch, module: types.ModuleType, mod: types.ModuleType):
    """Point every public function of `module` (and its re-export in the package) at `mod`'s."""
    for attr in dir(module):
        fn = getattr(module, attr)
        if attr.startswith("_") or not callable(fn) or getattr(fn, "__module__", None) != module.__name__:
            continue
        monkeypatch.setattr(module, attr, getattr(mod, attr))
        if module is hse_oracle and hasattr(oracle, attr):
            monkeypatch.setattr(oracle, attr, getattr(mod, attr))


def _caught(pins) -> bool:
    caught = False
    for pin in pins:
        try:
            pin()
        except AssertionError:
            caught = True
    return caught


CASES = ([(hse_oracle,) + m for m in MUTANTS] + [(oracle.tdks,) + m for m in TDKS_MUTANTS]
         + [(oracle.ortho,) + m for m in ORTHO_MUTANTS])


@pytest.mark.parametrize("module,name,old,new,pins", CASES, ids=[c[1] for c in CASES])
def test_pins_catch_planted_mistake(module, name, old, new, pins, monkeypatch):
    _install(monkeypatch, module, _load(module, old, new))
    assert _caught(pins), f"no pin caught the planted mistake: {name}"


@pytest.mark.parametrize("module", [hse_oracle, oracle.tdks, oracle.ortho], ids=lambda m: m.__name__)
def test_unmutated_copy_passes_the_same_pins(module, monkeypatch):
    """The harness itself: the unmodified source, loaded and installed the same way, passes
    every pin listed for the module."""
    _install(monkeypatch, module, _load(module, "import numpy as np\n", "import numpy as np\n"))
    seen = set()
    for case in CASES:
        if case[0] is not module:
            continue
        for pin in case[4]:
            if id(pin) not in seen:
                seen.add(id(pin))
                pin()
