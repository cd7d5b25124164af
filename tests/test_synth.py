"""The seeded input recipe, checked against the paper's workload shapes.

The generator builds cells, k-meshes, basis spheres, orbitals and occupations
and nothing else.  These tests pin each part of that recipe to something
independent of its code: closed forms of cell geometry, brute-force basis
enumeration, orthonormality, and the workload sizes of the paper's Table I
(grids doubled, Monkhorst-Pack meshes, the setup section's cutoff).
"""
import itertools
import math

import numpy as np
import pytest

from paper_1111_0716_gb300 import synth


@pytest.fixture(scope="module")
def beta():
    return synth.beta_boron()


@pytest.fixture(scope="module")
def alpha():
    return synth.alpha_boron()


@pytest.mark.parametrize("a,alpha_deg,omega", [(9.56, 58.06, 590.33), (19.17, 65.2, 5546.05)])
def test_rhombohedral_cells(a, alpha_deg, omega):
    """Equal edges and angles; volume from the closed form a^3 sqrt(1 - 3c^2 + 2c^3)."""
    lat = synth.rhombohedral_lattice(a, alpha_deg)
    assert np.allclose(np.linalg.norm(lat, axis=1), a, rtol=0, atol=1e-12)
    c = math.cos(math.radians(alpha_deg))
    for i, j in ((0, 1), (0, 2), (1, 2)):
        assert lat[i] @ lat[j] == pytest.approx(a * a * c, rel=1e-13)
    vol = abs(np.linalg.det(lat))
    assert vol == pytest.approx(a ** 3 * math.sqrt(1 - 3 * c * c + 2 * c ** 3), rel=1e-12)
    assert vol == pytest.approx(omega, abs=0.01)


@pytest.mark.parametrize("lat", [synth.cubic_lattice(10.0), synth.rhombohedral_lattice(9.56, 58.06)])
def test_reciprocal_rows(lat):
    """a_i . b_j = 2 pi delta_ij, with b_i from cross products (independent of the inverse)."""
    B = synth.reciprocal(lat)
    vol = lat[0] @ np.cross(lat[1], lat[2])
    cross = np.array([np.cross(lat[1], lat[2]), np.cross(lat[2], lat[0]), np.cross(lat[0], lat[1])])
    assert np.allclose(B, 2 * math.pi * cross / vol, rtol=0, atol=1e-13)
    assert np.allclose(lat @ B.T, 2 * math.pi * np.eye(3), rtol=0, atol=1e-12)


def test_k_meshes():
    """MP 4x4x4: fractions +-1/8, +-3/8; Gamma-centred 2x2x2: {0, 1/2}^3.  Both give the
    same set of k - q differences modulo 1 (multiples of 1/4), so the same kernel classes."""
    mp = synth.monkhorst_pack(4)
    assert mp.shape == (64, 3)
    assert set(np.unique(mp)) == {-3 / 8, -1 / 8, 1 / 8, 3 / 8}
    assert len({tuple(r) for r in mp}) == 64
    gc = synth.gamma_centred(2)
    assert {tuple(r) for r in gc} == set(itertools.product((0.0, 0.5), repeat=3))

    def diffs(mesh):
        d = (mesh[:, None, :] - mesh[None, :, :]).reshape(-1, 3) % 1.0
        return {tuple(np.round(r * 4).astype(int) % 4) for r in d}
    assert diffs(mp) == diffs(synth.gamma_centred(4)) == set(itertools.product(range(4), repeat=3))


@pytest.mark.parametrize("lat,kfrac,gcut", [
    (synth.cubic_lattice(10.0), np.zeros(3), math.pi),
    (synth.rhombohedral_lattice(9.56, 58.06), np.array([0.375, -0.125, 0.125]), 4.5),
    (synth.rhombohedral_lattice(19.17, 65.2), np.array([0.5, 0.0, 0.5]), 2.0),
])
def test_basis_sphere_is_complete_and_ordered(lat, kfrac, gcut):
    """Every Miller index with |(m + k) B| < gcut, found by brute force over a wide box,
    is in the basis, nothing else is, and the order is lexicographic."""
    m = synth.sphere_miller(lat, kfrac, gcut)
    B = synth.reciprocal(lat)
    # |m_i| <= |(m+k).B| |a_i| / 2pi + |k_i|: a box twice that wide is surely enough
    bound = int(math.ceil(2 * gcut * np.linalg.norm(lat, axis=1).max() / (2 * math.pi))) + 2
    want = []
    for t in itertools.product(range(-bound, bound + 1), repeat=3):
        g = (np.array(t) + kfrac) @ B
        if g @ g < gcut * gcut:
            want.append(t)
    assert [tuple(int(v) for v in r) for r in m] == want


def test_basis_sizes(alpha, beta):
    """Basis sizes of the paper-shaped cells at |G+k| < 4.5 and the tiny cubic cell."""
    assert synth.tiny_cubic().npw.tolist() == [485]
    assert alpha.npw.min() == 897 and alpha.npw.max() == 924
    assert beta.npw.min() == 8540 and beta.npw.max() == 8548
    assert [int(synth.plane_wave_cell(s).npw[0]) for s in synth.PW_SHELLS] == [19, 57, 81, 179]


@pytest.mark.parametrize("make", [synth.tiny_cubic, synth.alpha_boron, lambda: synth.sweep_cell(2)])
def test_orbitals_orthonormal_and_zero_padded(make):
    wl = make()
    for k in range(wl.nk):
        n = int(wl.npw[k])
        c = wl.coeff[k, :, :n]
        assert np.abs(c.conj() @ c.T - np.eye(c.shape[0])).max() < 1e-13
        assert not wl.coeff[k, :, n:].any()
        assert not wl.miller[k, n:].any()


def test_orbitals_are_band_limited_by_the_envelope(alpha):
    """Amplitudes carry exp(-|G+k|^2/8), so the band-averaged weight |c|^2 falls as
    exp(-|G+k|^2/4): the slope of its logarithm against |G+k|^2 is -1/4 (orthonormalising
    18 bands in a ~900-function basis barely changes it)."""
    B = synth.reciprocal(alpha.lattice)
    g2, p = [], []
    for k in range(alpha.nk):
        n = int(alpha.npw[k])
        g2.append((((alpha.miller[k, :n] + alpha.kfrac[k]) @ B) ** 2).sum(axis=1))
        p.append((np.abs(alpha.coeff[k, :, :n]) ** 2).mean(axis=0))
    slope = np.polyfit(np.concatenate(g2), np.log(np.concatenate(p)), 1)[0]
    assert -0.27 < slope < -0.23


def test_seeded_and_reproducible():
    a, b = synth.tiny_cubic(seed=1), synth.tiny_cubic(seed=1)
    assert np.array_equal(a.coeff, b.coeff)
    assert not np.array_equal(a.coeff, synth.tiny_cubic(seed=2).coeff)


def test_occupations(beta):
    """beta cell: w = 1 for bands 1-150, 0.5 for 151-160, 0 for targets 161-192."""
    assert beta.n_occ == 160 and beta.n_tgt == 192
    assert (beta.w[:, :150] == 1.0).all()
    assert (beta.w[:, 150:160] == 0.5).all()
    assert (beta.w[:, 160:] == 0.0).all()
    tiny = synth.tiny_cubic()
    assert (tiny.w == 1.0).all()


def test_grids_admit_the_codensity_without_aliasing(beta):
    """Every workload's grid satisfies N >= 4 n_max + 1 on each axis."""
    for wl in [synth.tiny_cubic(), synth.alpha_boron(), beta, synth.differentiation_cell()] + \
            [synth.sweep_cell(i) for i in range(len(synth.SWEEP_GRIDS))]:
        assert (np.array(wl.grid) >= 4 * wl.n_max() + 1).all(), wl.name
    assert beta.n_max().tolist() == [14, 14, 14]


def test_pair_counts(alpha, beta):
    """Logical band-pair applications per operator pass."""
    assert synth.tiny_cubic().pair_count() == 64
    assert alpha.pair_count() == 64 * 24 * 64 * 18 == 1769472
    assert beta.pair_count() == 8 * 192 * 8 * 160 == 1966080
    assert synth.differentiation_cell().pair_count() == 1024
    assert sum(synth.sweep_cell(i).pair_count() for i in range(6)) == 17472
