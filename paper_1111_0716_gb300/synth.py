"""Seeded synthetic workloads for the plane-wave Fock exchange operator.

This module only builds inputs: cells, k-meshes, plane-wave basis sets (Miller
indices inside a cutoff sphere), band-limited random orbitals and occupations.
It holds none of the exchange arithmetic (no codensities, no FFTs, no Coulomb
kernel), so it can feed both the CUDA library and the independent CPU oracle.

The shapes follow the paper's boron workloads (Table I: FFT grids of 24 and 48
points per axis, Monkhorst-Pack k-meshes; Sec. "Setup of DFT calculations":
319 eV plane-wave cutoff, i.e. |G+k| < 4.84 bohr^-1, here 4.5).  The paper's
atomic structures and PAW data are not available, so seeded band-limited random
orbitals stand in for the Kohn-Sham orbitals with the same basis sizes.

Conventions (Hartree atomic units, lengths in bohr):
  * lattice rows are a1, a2, a3; reciprocal rows b_i satisfy a_i . b_j = 2 pi d_ij;
  * a plane wave of Miller index m at k-point k has wavevector (m + k_frac) . B;
  * orbital coefficients c[k][b][g] are orthonormal per k: sum_g c_a* c_b = d_ab;
  * occupations w[k][b] are per spin, in [0, 1]; spin-paired (s = 2).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

KERNEL_HSE = 0          # screened erfc(mu r)/r interaction
KERNEL_COULOMB = 1      # bare 1/r interaction with the g = 0 term dropped

HSE06_MU = 0.106        # bohr^-1 (0.2 Angstrom^-1)


@dataclasses.dataclass
class Workload:
    """One exchange problem: cell, grid, k-mesh, basis, orbitals, occupations."""
    name: str
    lattice: np.ndarray          # (3, 3) float64, rows a1, a2, a3
    grid: tuple                  # (N1, N2, N3)
    kfrac: np.ndarray            # (nk, 3) float64, fractional k-points
    npw: np.ndarray              # (nk,) int32, basis size per k
    miller: np.ndarray           # (nk, npw_max, 3) int32, zero padded
    coeff: np.ndarray            # (nk, nb, npw_max) complex128, zero padded
    w: np.ndarray                # (nk, nb) float64 per-spin occupations
    n_occ: int                   # occupied bands are coeff[:, :n_occ]
    n_tgt: int                   # target bands are coeff[:, :n_tgt]
    kernel: int = KERNEL_HSE
    mu: float = HSE06_MU
    seed: Optional[int] = None

    @property
    def nk(self) -> int:
        return int(self.kfrac.shape[0])

    @property
    def npw_max(self) -> int:
        return int(self.miller.shape[1])

    @property
    def c_occ(self) -> np.ndarray:
        return np.ascontiguousarray(self.coeff[:, :self.n_occ])

    @property
    def c_tgt(self) -> np.ndarray:
        return np.ascontiguousarray(self.coeff[:, :self.n_tgt])

    @property
    def w_occ(self) -> np.ndarray:
        return np.ascontiguousarray(self.w[:, :self.n_occ])

    @property
    def w_tgt(self) -> np.ndarray:
        return np.ascontiguousarray(self.w[:, :self.n_tgt])

    def n_max(self) -> np.ndarray:
        """Largest |Miller index| per axis over every basis set."""
        out = np.zeros(3, dtype=np.int64)
        for k in range(self.nk):
            m = self.miller[k, :self.npw[k]]
            out = np.maximum(out, np.abs(m).max(axis=0))
        return out

    def pair_count(self) -> int:
        """Logical (k, a, q, j) band-pair applications in one operator pass."""
        return self.nk * self.n_tgt * self.nk * self.n_occ

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


# ---------------------------------------------------------------- geometry

def cubic_lattice(L: float) -> np.ndarray:
    return np.diag([L, L, L]).astype(np.float64)


def rhombohedral_lattice(a: float, alpha_deg: float) -> np.ndarray:
    """Rhombohedral cell with |a_i| = a and all inter-axis angles alpha.

    a1 along x, a2 in the xy plane, a3 completes the rhombohedron.  Any
    orientation gives the same exchange energy (rotation invariance).
    """
    ca = math.cos(math.radians(alpha_deg))
    sa = math.sin(math.radians(alpha_deg))
    a1 = [1.0, 0.0, 0.0]
    a2 = [ca, sa, 0.0]
    cy = (ca - ca * ca) / sa
    cz = math.sqrt(max(0.0, 1.0 - ca * ca - cy * cy))
    a3 = [ca, cy, cz]
    return a * np.array([a1, a2, a3], dtype=np.float64)


def reciprocal(lattice: np.ndarray) -> np.ndarray:
    """Rows b_i with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * math.pi * np.linalg.inv(lattice).T


def monkhorst_pack(n: int) -> np.ndarray:
    """Full n x n x n Monkhorst-Pack mesh, fractions (2r - n - 1) / (2n)."""
    f = [(2 * r - n - 1) / (2.0 * n) for r in range(1, n + 1)]
    return np.array([[a, b, c] for a in f for b in f for c in f], dtype=np.float64)


def gamma_centred(n: int) -> np.ndarray:
    """Full Gamma-centred n x n x n mesh, fractions r / n for r = 0..n-1."""
    f = [r / float(n) for r in range(n)]
    return np.array([[a, b, c] for a in f for b in f for c in f], dtype=np.float64)


def sphere_miller(lattice: np.ndarray, kfrac: np.ndarray, gcut: float) -> np.ndarray:
    """Miller indices m with |(m + k) . B| < gcut, in lexicographic (m1, m2, m3) order."""
    B = reciprocal(lattice)
    lens = np.linalg.norm(lattice, axis=1)
    bound = [int(math.ceil(gcut * lens[i] / (2.0 * math.pi) + abs(kfrac[i]))) + 1
             for i in range(3)]
    r = [np.arange(-bound[i], bound[i] + 1) for i in range(3)]
    m = np.stack(np.meshgrid(r[0], r[1], r[2], indexing="ij"), axis=-1).reshape(-1, 3)
    g = (m + kfrac[None, :]) @ B
    keep = np.einsum("ij,ij->i", g, g) < gcut * gcut
    return m[keep].astype(np.int32)          # meshgrid 'ij' order is lexicographic


def _basis(lattice, kfrac, gcut):
    sets = [sphere_miller(lattice, kfrac[k], gcut) for k in range(kfrac.shape[0])]
    npw = np.array([s.shape[0] for s in sets], dtype=np.int32)
    miller = np.zeros((len(sets), int(npw.max()), 3), dtype=np.int32)
    for k, s in enumerate(sets):
        miller[k, :s.shape[0]] = s
    return npw, miller


def orthonormalise(m: np.ndarray) -> np.ndarray:
    """Gram-Schmidt of the columns of m (npw x nb) in column order, FP64.

    Computed through a Householder QR followed by a phase fix that makes the
    diagonal of R real positive; that factorisation is unique, so the columns
    equal those of (modified) Gram-Schmidt in exact arithmetic.
    """
    q, r = np.linalg.qr(m)
    d = np.diag(r)
    ph = d / np.abs(d)
    return q * ph[None, :]


def random_orbitals(rng: np.random.Generator, lattice, kfrac, npw, miller, nb,
                    envelope: float = 8.0) -> np.ndarray:
    """Band-limited complex Gaussian orbitals, orthonormal per k.

    Draw order: k, band, G (lexicographic Miller order); real and imaginary
    parts iid N(0, 1); envelope exp(-|G+k|^2 / envelope).
    """
    B = reciprocal(lattice)
    nk = kfrac.shape[0]
    out = np.zeros((nk, nb, miller.shape[1]), dtype=np.complex128)
    for k in range(nk):
        n = int(npw[k])
        if nb > n:
            raise ValueError("more bands than plane waves")
        z = rng.standard_normal((nb, n, 2))
        c = z[..., 0] + 1j * z[..., 1]
        g = (miller[k, :n] + kfrac[k][None, :]) @ B
        c *= np.exp(-np.einsum("ij,ij->i", g, g) / envelope)[None, :]
        out[k, :, :n] = orthonormalise(c.T).T
    return out


def minus_g_index(miller: np.ndarray) -> np.ndarray:
    """Row of -m for every Miller row m of one basis set (ValueError if one is missing)."""
    pos = {tuple(int(v) for v in m): i for i, m in enumerate(miller)}
    try:
        return np.array([pos[tuple(-int(v) for v in m)] for m in miller], dtype=np.int64)
    except KeyError:
        raise ValueError("basis set is not closed under G -> -G") from None


def random_real_orbitals(rng: np.random.Generator, lattice, npw, miller, nb,
                         envelope: float = 8.0) -> np.ndarray:
    """Gamma-point orbitals that are real in real space, orthonormal: c(-G) = conj c(G).

    Each orbital is drawn as real coefficients x on the real basis {1 at G = 0;
    sqrt2 cos(G.r), sqrt2 sin(G.r) for each pair (G, -G) with G's first nonzero
    Miller component positive}, iid N(0, 1) times the envelope, orthonormalised
    (QR in real arithmetic, diagonal of R positive), then mapped to plane waves by
    c(G) = (x_cos - i x_sin)/sqrt2, c(-G) = (x_cos + i x_sin)/sqrt2, c(0) = x_0.
    The map is unitary, so orthonormal x give orthonormal c.  Draw order: band,
    then real basis function in lexicographic order of G (cos before sin).
    """
    B = reciprocal(lattice)
    n = int(npw[0])
    if nb > n:
        raise ValueError("more bands than plane waves")
    m = miller[0, :n]
    neg = minus_g_index(m)
    first = np.array([next((int(v) for v in row if v != 0), 0) for row in m])
    zero = np.flatnonzero(first == 0)
    pos = np.flatnonzero(first > 0)
    g = m @ B
    env = np.exp(-np.einsum("ij,ij->i", g, g) / envelope)
    # real basis functions in lexicographic order of their G: G = 0 (if present), then pairs
    scale = np.concatenate([env[zero], np.repeat(env[pos], 2)])
    x = rng.standard_normal((nb, scale.size)) * scale[None, :]
    q, r = np.linalg.qr(x.T)
    q = q * np.sign(np.diag(r))[None, :]
    x = q.T                                            # (nb, n) orthonormal rows
    out = np.zeros((1, nb, miller.shape[1]), dtype=np.complex128)
    nz = zero.size
    out[0][:, zero] = x[:, :nz]
    xc, xs = x[:, nz::2], x[:, nz + 1::2]
    out[0][:, pos] = (xc - 1j * xs) / math.sqrt(2.0)
    out[0][:, neg[pos]] = (xc + 1j * xs) / math.sqrt(2.0)
    return out


def make_workload(name, lattice, grid, kfrac, gcut, n_occ, n_tgt, w_occ_values,
                  seed, kernel=KERNEL_HSE, mu=HSE06_MU, real=False) -> Workload:
    rng = np.random.Generator(np.random.PCG64(seed))
    npw, miller = _basis(lattice, kfrac, gcut)
    nb = max(n_occ, n_tgt)
    if real:
        if kfrac.shape[0] != 1 or np.any(kfrac != 0.0):
            raise ValueError("real orbitals need a Gamma-only mesh")
        coeff = random_real_orbitals(rng, lattice, npw, miller, nb)
    else:
        coeff = random_orbitals(rng, lattice, kfrac, npw, miller, nb)
    w = np.zeros((kfrac.shape[0], nb), dtype=np.float64)
    w[:, :n_occ] = np.asarray(w_occ_values, dtype=np.float64)[None, :]
    return Workload(name=name, lattice=lattice, grid=tuple(int(g) for g in grid),
                    kfrac=np.ascontiguousarray(kfrac, dtype=np.float64), npw=npw,
                    miller=miller, coeff=coeff, w=w, n_occ=n_occ, n_tgt=n_tgt,
                    kernel=kernel, mu=mu, seed=seed)


# ---------------------------------------------------------------- workloads

def tiny_cubic(seed: int = 1, grid: int = 24, nb: int = 8, kernel=KERNEL_HSE) -> Workload:
    """Cubic L = 10 bohr, Gamma only, |G| < 5 (2 pi / L), nb doubly occupied bands."""
    L = 10.0
    return make_workload("cubic-L10-%d^3-%db" % (grid, nb), cubic_lattice(L), (grid,) * 3,
                         np.zeros((1, 3)), 5.0 * 2.0 * math.pi / L, nb, nb,
                         [1.0] * nb, seed, kernel=kernel)


def alpha_boron(seed: int = 2, mesh: int = 4) -> Workload:
    """alpha-boron-sized rhombohedral cell (12 atoms' worth), 48^3, MP mesh."""
    return make_workload("alpha-B12-48^3-MP%d" % mesh, rhombohedral_lattice(9.56, 58.06),
                         (48,) * 3, monkhorst_pack(mesh), 4.5, 18, 24, [1.0] * 18, seed)


def beta_boron(seed: int = 3, mesh: int = 2) -> Workload:
    """beta-boron-sized rhombohedral cell (~106 atoms' worth), 96^3, Gamma-centred mesh.

    160 occupied bands (w = 1 for bands 1-150, 0.5 for 151-160), 192 targets.
    """
    w = [1.0] * 150 + [0.5] * 10
    return make_workload("beta-B106-96^3-G%d" % mesh, rhombohedral_lattice(19.17, 65.2),
                         (96,) * 3, gamma_centred(mesh), 4.5, 160, 192, w, seed)


def differentiation_cell(seed: int = 4) -> Workload:
    """The tiny cubic cell at 48^3 with 32 occupied bands (targets = occupied)."""
    return tiny_cubic(seed=seed, grid=48, nb=32)


SWEEP_GRIDS = (32, 40, 48, 60, 72, 80)
SWEEP_BANDS = (16, 24, 32, 48, 64, 96)


def sweep_cell(i: int, kernel=KERNEL_HSE) -> Workload:
    """Cell i of the uneven precision sweep: cubic L = 10 N / 24, same cutoff as tiny_cubic."""
    n, nb = SWEEP_GRIDS[i], SWEEP_BANDS[i]
    L = 10.0 * n / 24.0
    return make_workload("sweep-%d^3-%db-%s" % (n, nb, "hse" if kernel == KERNEL_HSE else "coul"),
                         cubic_lattice(L), (n,) * 3, np.zeros((1, 3)), math.pi, nb, nb,
                         [1.0] * nb, 51 + i, kernel=kernel)


PW_SHELLS = (2, 5, 6, 12)


def plane_wave_cell(shell: int, grid: int = 32, L: float = 10.0) -> Workload:
    """Cubic cell whose occupied orbitals are single plane waves exp(iG.r)/sqrt(Omega).

    The basis is every Miller index with |m|^2 <= shell; orbital b is the unit
    vector on basis function b.  Bare Coulomb kernel, w = 1.
    """
    r = np.arange(-4, 5)
    m = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    m = m[(m * m).sum(axis=1) <= shell].astype(np.int32)
    n = m.shape[0]
    coeff = np.eye(n, dtype=np.complex128)[None]
    return Workload(name="pw-shell%d-%d^3" % (shell, grid), lattice=cubic_lattice(L),
                    grid=(grid,) * 3, kfrac=np.zeros((1, 3)),
                    npw=np.array([n], dtype=np.int32), miller=m[None].copy(),
                    coeff=coeff, w=np.ones((1, n)), n_occ=n, n_tgt=n,
                    kernel=KERNEL_COULOMB, mu=0.0, seed=None)


def real_tiny_cubic(seed: int = 61, grid: int = 24, n_occ: int = 7, n_tgt: int = 9,
                    kernel=KERNEL_HSE) -> Workload:
    """tiny_cubic with real (Gamma-point) orbitals, an odd occupied count and extra targets."""
    L = 10.0
    w = [1.0] * (n_occ - 1) + [0.5]
    return make_workload("real-cubic-L10-%d^3-%do-%dt" % (grid, n_occ, n_tgt), cubic_lattice(L),
                         (grid,) * 3, np.zeros((1, 3)), 5.0 * 2.0 * math.pi / L, n_occ, n_tgt,
                         w, seed, kernel=kernel, real=True)


def real_alpha_cell(seed: int = 62) -> Workload:
    """alpha-boron-sized rhombohedral cell at Gamma only, 48^3, real orbitals, 18 occ / 24 tgt."""
    return make_workload("real-alpha-B12-48^3-G", rhombohedral_lattice(9.56, 58.06), (48,) * 3,
                         np.zeros((1, 3)), 4.5, 18, 24, [1.0] * 16 + [0.5] * 2, seed, real=True)


def real_beta_cell(seed: int = 63) -> Workload:
    """beta-boron-sized rhombohedral cell at Gamma only, 96^3, real orbitals, 160 occ / 192 tgt."""
    w = [1.0] * 150 + [0.5] * 10
    return make_workload("real-beta-B106-96^3-G", rhombohedral_lattice(19.17, 65.2), (96,) * 3,
                         np.zeros((1, 3)), 4.5, 160, 192, w, seed, real=True)


def all_parity_workloads() -> List[Workload]:
    return [tiny_cubic(), alpha_boron(), beta_boron(), differentiation_cell()] + \
        [sweep_cell(i) for i in range(len(SWEEP_GRIDS))]
