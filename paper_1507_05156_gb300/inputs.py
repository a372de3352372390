"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only *generates* data: cells, Monkhorst-Pack k-meshes, occupations and
orthonormal Bloch orbitals.  It contains none of the exchange operator's arithmetic
(no pair densities, no screened kernel, no accumulation), so both sides of every
parity check can take their inputs from here without sharing any of the method.

Recipe (synthetic stand-in for the paper's silicon runs, Sec. II C: an 8-atom cubic
cell, a 16^3 real-space grid and 16 occupied bands; no pseudopotential data is used):

* cell: simple cubic, lattice constant a = 10.26 bohr (rows a1, a2, a3 of ``lattice``);
* k-mesh: Monkhorst-Pack, k = sum_d (2 r_d - n_d - 1) / (2 n_d) b_d, r_d = 1..n_d,
  in Cartesian bohr^-1, r_1 slowest;
* orbitals: for every k and band, plane-wave coefficients c(G) drawn i.i.d. complex
  standard normal for |G + k|^2 / 2 < ecut (6 Ha), u(r) = sum_G c(G) e^{i G.r} on the
  grid, then Gram-Schmidt orthonormalised per k in the cell inner product
  <a|b> = dV sum_r conj(a(r)) b(r), dV = Omega / N, so that dV sum_r |u|^2 = 1;
* occupations f = 1 for occupied bands.

Layout of every orbital array: [nk][nbands][N1][N2][N3], C order, z (N3) fastest,
complex.  Grid index (i1, i2, i3) is the point r = i1/N1 a1 + i2/N2 a2 + i3/N3 a3.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903

#: Lattice constant of the synthetic silicon-like cubic cell (bohr).
A_SI = 10.26
#: Screening parameter used by the workloads (bohr^-1).
OMEGA = 0.106
#: Screening parameter the paper quotes, 0.3 1/angstrom, in bohr^-1 (Sec. II B).
OMEGA_PAPER = 0.3 / BOHR_PER_ANGSTROM
#: Fock mixing fraction of HSE (Sec. II B).
ALPHA = 0.25
#: Plane-wave cutoff of the random orbitals (Ha).
ECUT = 6.0
#: Base seed of the workloads; workload w uses SEED_BASE + w.
SEED_BASE = 1507051560


def cubic_lattice(a: float = A_SI) -> np.ndarray:
    """Rows a1, a2, a3 of a simple cubic cell of side ``a`` (bohr)."""
    return np.eye(3) * float(a)


def _reciprocal_rows(lattice: np.ndarray) -> np.ndarray:
    # b_i . a_j = 2 pi delta_ij; rows b1, b2, b3.  Used only to place the random
    # plane-wave coefficients inside the cutoff sphere and to build the k-mesh.
    return 2.0 * np.pi * np.linalg.inv(np.asarray(lattice, dtype=np.float64)).T


def monkhorst_pack(n: tuple, lattice: np.ndarray) -> np.ndarray:
    """Cartesian Monkhorst-Pack k-points [n1*n2*n3][3] (bohr^-1), r_1 slowest."""
    b = _reciprocal_rows(lattice)
    fr = []
    for nd in n:
        fr.append([(2.0 * r - nd - 1.0) / (2.0 * nd) for r in range(1, nd + 1)])
    pts = []
    for f1 in fr[0]:
        for f2 in fr[1]:
            for f3 in fr[2]:
                pts.append(f1 * b[0] + f2 * b[1] + f3 * b[2])
    return np.array(pts, dtype=np.float64)


def monkhorst_pack_subset(n: tuple, m: tuple) -> np.ndarray:
    """Indices, in the ordering of monkhorst_pack(n), of the points of the coarser mesh
    monkhorst_pack(m) (the q-point sub-mesh of the down-sampled Fock sum).  Each n_d must be
    an odd multiple s_d of m_d, which makes the coarse mesh an exact subset: along axis d the
    coarse points are the fine points r = s_d r' + (s_d - 1)/2 (0-based)."""
    axes = []
    for nd, md in zip(n, m):
        if md < 1 or nd % md or (nd // md) % 2 == 0:
            raise ValueError("each fine mesh side must be an odd multiple of the coarse one")
        s = nd // md
        axes.append([s * r + (s - 1) // 2 for r in range(md)])
    return np.array([(r1 * n[1] + r2) * n[2] + r3 for r1 in axes[0] for r2 in axes[1] for r3 in axes[2]],
                    dtype=np.int64)


def _fft_order(nd: int) -> np.ndarray:
    # integer frequency of array index 0..nd-1 (numpy fftfreq order)
    return np.fft.fftfreq(nd, d=1.0 / nd).round().astype(np.int64)


def orthonormal_orbitals(rng: np.random.Generator, grid: tuple, lattice: np.ndarray,
                         kpts: np.ndarray, nbands: int, ecut: float = ECUT) -> np.ndarray:
    """Random cell-normalised, per-k orthonormal periodic orbitals u_{b,k}(r).

    Returns complex128 [nk][nbands][N1][N2][N3].
    """
    n1, n2, n3 = (int(g) for g in grid)
    N = n1 * n2 * n3
    b = _reciprocal_rows(lattice)
    omega_cell = abs(np.linalg.det(lattice))
    dV = omega_cell / N
    m1, m2, m3 = np.meshgrid(_fft_order(n1), _fft_order(n2), _fft_order(n3), indexing="ij")
    Gc = (m1[..., None] * b[0] + m2[..., None] * b[1] + m3[..., None] * b[2])
    nk = len(kpts)
    out = np.empty((nk, nbands, n1, n2, n3), dtype=np.complex128)
    for ik in range(nk):
        kin = 0.5 * np.sum((Gc + kpts[ik]) ** 2, axis=-1)
        mask = kin < ecut
        npw = int(mask.sum())
        if npw < nbands:
            raise ValueError(f"cutoff sphere holds {npw} plane waves < {nbands} bands")
        coef = np.zeros((nbands, n1, n2, n3), dtype=np.complex128)
        draw = (rng.standard_normal((nbands, npw)) + 1j * rng.standard_normal((nbands, npw))) / np.sqrt(2.0)
        coef[:, mask] = draw
        # u(r) = sum_G c(G) e^{i G.r}: an unnormalised inverse transform of the grid
        u = np.fft.ifftn(coef, axes=(1, 2, 3)) * N
        out[ik] = u
    return gram_schmidt(out, dV)


def gram_schmidt(u: np.ndarray, dV: float) -> np.ndarray:
    """Orthonormalise the bands of every k in <a|b> = dV sum conj(a) b.

    Gram-Schmidt in band order, computed as a Householder QR factorisation with the
    phases fixed so that R has a positive real diagonal: that is exactly the set of
    vectors classical Gram-Schmidt produces, with better rounding.
    """
    nk, nb = u.shape[:2]
    flat = u.reshape(nk, nb, -1)
    A = np.transpose(flat, (0, 2, 1))  # [nk][N][nb]
    Q, R = np.linalg.qr(A)
    d = np.diagonal(R, axis1=1, axis2=2)
    ph = d / np.abs(d)
    Q = Q * ph[:, None, :]
    out = np.transpose(Q, (0, 2, 1)).reshape(u.shape) / np.sqrt(dV)
    return np.ascontiguousarray(out)


@dataclasses.dataclass
class Cell:
    """One exchange problem: a cell, its k-mesh and orbitals (all FP64 / complex128)."""

    name: str
    grid: tuple
    lattice: np.ndarray
    kpts: np.ndarray          # [nk][3] Cartesian bohr^-1
    u_occ: np.ndarray         # [nk][n_occ][N1][N2][N3] complex128
    occ: np.ndarray           # [nk][n_occ] float64
    u_tgt: np.ndarray         # [nk][n_tgt][N1][N2][N3] complex128
    omega: float = OMEGA
    alpha: float = ALPHA
    spin_degeneracy: float = 2.0
    tgt_is_occ: bool = True   # u_tgt holds exactly the occupied set

    @property
    def nk(self) -> int:
        return int(self.kpts.shape[0])

    @property
    def n_occ(self) -> int:
        return int(self.u_occ.shape[1])

    @property
    def n_tgt(self) -> int:
        return int(self.u_tgt.shape[1])

    @property
    def npts(self) -> int:
        return int(np.prod(self.grid))

    @property
    def pairs(self) -> int:
        """Ordered (i,k; j,k') pair convolutions in one Fock apply."""
        return self.nk * self.n_tgt * self.nk * self.n_occ


def make_cell(seed: int, grid: tuple, kmesh: tuple, n_occ: int, n_empty: int = 0,
              a: float = A_SI, omega: float = OMEGA, alpha: float = ALPHA,
              name: str = "cell") -> Cell:
    """A seeded cell: orbitals for n_occ + n_empty bands, targets = all of them."""
    rng = np.random.default_rng(seed)
    lattice = cubic_lattice(a)
    kpts = monkhorst_pack(tuple(kmesh), lattice)
    u = orthonormal_orbitals(rng, tuple(grid), lattice, kpts, n_occ + n_empty)
    u_occ = np.ascontiguousarray(u[:, :n_occ])
    occ = np.ones((len(kpts), n_occ), dtype=np.float64)
    return Cell(name=name, grid=tuple(int(g) for g in grid), lattice=lattice, kpts=kpts,
                u_occ=u_occ, occ=occ, u_tgt=u, omega=omega, alpha=alpha,
                tgt_is_occ=(n_empty == 0))


# ---------------------------------------------------------------------------
# The five workloads.  Index w is the workload number used for the seed.
# ---------------------------------------------------------------------------

WORKLOADS = {
    0: dict(name="fp64_12cube_k2_b4", grid=(12, 12, 12), kmesh=(2, 2, 2), n_occ=4, n_empty=0),
    1: dict(name="c64_20cube_k4_b16", grid=(20, 20, 20), kmesh=(4, 4, 4), n_occ=16, n_empty=0),
    2: dict(name="c64_24cube_k8_b16+16", grid=(24, 24, 24), kmesh=(8, 8, 8), n_occ=16, n_empty=16),
    4: dict(name="diff_16cube_k3_b8", grid=(16, 16, 16), kmesh=(3, 3, 3), n_occ=8, n_empty=0),
}

BATCHED_GRIDS = (12, 16, 18, 20, 24)
BATCHED_KMESH = (2, 3, 4)


def workload(w: int) -> Cell:
    """Workload ``w`` (0, 1, 2 or 4); workload 3 is the batched list, see batched_cells."""
    spec = WORKLOADS[w]
    return make_cell(SEED_BASE + w, spec["grid"], spec["kmesh"], spec["n_occ"], spec["n_empty"],
                     name=spec["name"])


def batched_specs(ncells: int = 32, seed: Optional[int] = None) -> List[dict]:
    """Draw the uneven batch: grid from {12,16,18,20,24}^3, n^3 k-mesh n in {2,3,4},
    4..16 bands with n_tgt = n_occ; one sub-seed per cell."""
    seed = SEED_BASE + 3 if seed is None else seed
    rng = np.random.default_rng(seed)
    specs = []
    for c in range(ncells):
        g = int(rng.choice(BATCHED_GRIDS))
        n = int(rng.choice(BATCHED_KMESH))
        nb = int(rng.integers(4, 17))
        specs.append(dict(name=f"cell{c:02d}_{g}cube_k{n}_b{nb}", grid=(g, g, g), kmesh=(n, n, n),
                          n_occ=nb, n_empty=0, seed=int(rng.integers(0, 2**31 - 1))))
    return specs


def batched_cells(ncells: int = 32, seed: Optional[int] = None) -> List[Cell]:
    return [make_cell(s["seed"], s["grid"], s["kmesh"], s["n_occ"], s["n_empty"], name=s["name"])
            for s in batched_specs(ncells, seed)]


def random_orbitals(seed: int, shape: tuple) -> np.ndarray:
    """Plain seeded complex normal array (cotangents, perturbation directions)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
