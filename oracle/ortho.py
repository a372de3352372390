"""FP64 CPU oracle of the orbital overlap and Gram-Schmidt orthonormalisation (test
infrastructure: only ``tests/`` may use it).

The orbitals u_{b,k} of the method are cell-normalised, <a|b> = dV sum_r conj(u_a(r)) u_b(r)
with dV = Omega / N (Sec. II C works with orthonormal Bloch orbitals; the 4th-order Taylor
propagator of Sec. II C is not unitary, so the drift of the overlap from the identity is
the check of a propagation).

* overlap: S[k][a][b] = dV sum_r conj(u_{a,k}(r)) u_{b,k}(r), plain FP64 sums.
* gram_schmidt: modified Gram-Schmidt per k-point in band order -- for each band a, subtract
  its component along every earlier (already orthonormal) band b < a, one at a time, then
  divide by its norm -- applied twice (the second pass removes what rounding left of the
  projections), all in FP64.
"""
from __future__ import annotations

import numpy as np


def overlap(u, dV: float) -> np.ndarray:
    """S [nk][nb][nb] complex128 of u [nk][nb][...]."""
    u = np.asarray(u, dtype=np.complex128)
    v = u.reshape(u.shape[0], u.shape[1], -1)
    return dV * np.einsum("kar,kbr->kab", np.conj(v), v)


def gram_schmidt(u, dV: float, passes: int = 2) -> np.ndarray:
    """Orthonormalised copy of u [nk][nb][...] (modified Gram-Schmidt, ``passes`` times)."""
    u = np.array(u, dtype=np.complex128)
    shape = u.shape
    v = u.reshape(shape[0], shape[1], -1)
    for _ in range(passes):
        for k in range(v.shape[0]):
            for a in range(v.shape[1]):
                for b in range(a):
                    v[k, a] -= (dV * np.vdot(v[k, b], v[k, a])) * v[k, b]
                v[k, a] /= np.sqrt(dV * np.vdot(v[k, a], v[k, a]).real)
    return v.reshape(shape)
