"""Pins of the FP64 CPU oracle against mathematics it does not itself use.

Each test ties one part of the oracle to something independent of its code:
the DFT definition, numpy's FFT, a numerical Fourier integral of the screened
interaction, a brute-force real-space convolution, a grid-free coefficient-space
double convolution, exact plane-wave lattice sums and the Dirac exchange of the
homogeneous electron gas, symmetry invariances and finite differences.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from paper_1111_0716_gb300 import synth
from tests import coeffspace


# ------------------------------------------------------------------ helpers

def direct_dft3(x, sign):
    """O(N^2) DFT straight from the definition, over flattened (i3, i2, i1)."""
    n3, n2, n1 = x.shape
    i3, i2, i1 = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    ph = (np.outer(i1.ravel(), i1.ravel()) / n1 + np.outer(i2.ravel(), i2.ravel()) / n2 +
          np.outer(i3.ravel(), i3.ravel()) / n3)
    return (np.exp(sign * 2j * math.pi * ph) @ x.ravel()).reshape(x.shape)


def rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def small_cubic(seed=11, grid=12, nb=6, kernel=synth.KERNEL_HSE, L=6.0, ncut=2.5):
    return synth.make_workload("small-cubic", synth.cubic_lattice(L), (grid,) * 3,
                               np.zeros((1, 3)), ncut * 2 * math.pi / L, nb, nb, [1.0] * nb,
                               seed, kernel=kernel)


def small_rhombo(seed=12, grid=16, kernel=synth.KERNEL_HSE):
    """Rhombohedral cell with a 2x2x2 Monkhorst-Pack mesh and fractional occupations."""
    wl = synth.make_workload("small-rhombo", synth.rhombohedral_lattice(7.0, 65.0), (grid,) * 3,
                             synth.monkhorst_pack(2), 2.0, 4, 5, [1.0, 1.0, 0.7, 0.25], seed,
                             kernel=kernel)
    assert np.all(4 * wl.n_max() + 1 <= grid)
    return wl


# ---------------------------------------------------------------------- FFT

@pytest.mark.parametrize("shape", [(6, 6, 6), (8, 8, 8), (10, 10, 10), (12, 12, 12), (15, 6, 10)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_direct_dft(oracle_mod, shape, sign):
    x = rand_c(np.random.default_rng(sum(shape)), shape)
    ref = direct_dft3(x, sign)
    got = oracle_mod.fft3d(x, sign)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n", [24, 32, 36, 40, 48, 54, 60, 64, 72, 80, 96, 108])
def test_fft_matches_numpy_on_every_grid_length(oracle_mod, n):
    x = rand_c(np.random.default_rng(n), (3, 5, n))
    ref = np.fft.fftn(x)
    got = oracle_mod.fft3d(x, -1)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max() * math.log2(x.size)
    inv = oracle_mod.fft3d(x, +1)
    ref_i = np.fft.ifftn(x) * x.size
    assert np.abs(inv - ref_i).max() <= 1e-13 * np.abs(ref_i).max() * math.log2(x.size)


def test_fft_parseval_on_codensity(oracle_mod):
    rng = np.random.default_rng(3)
    rho = rand_c(rng, (24, 24, 24))
    rh = oracle_mod.fft3d(rho, -1) / rho.size
    assert abs(np.mean(np.abs(rho) ** 2) - np.sum(np.abs(rh) ** 2)) <= 1e-13 * np.mean(np.abs(rho) ** 2)


# ------------------------------------------------------------------- kernel

@pytest.mark.parametrize("mu", [0.106, 0.4])
def test_screened_kernel_is_fourier_transform_of_erfc(oracle_mod, mu):
    """v(g) = int d^3r exp(-i g.r) erfc(mu r)/r, by 1D quadrature (QAWF)."""
    lat = synth.cubic_lattice(10.0)
    grid = (6, 6, 6)
    d = np.array([0.25, -0.125, 0.5])
    v = oracle_mod.kernel_grid(lat, grid, d, synth.KERNEL_HSE, mu)
    B = coeffspace.reciprocal(lat)
    for (i1, i2, i3) in [(0, 0, 0), (1, 0, 0), (2, 5, 1), (3, 3, 4)]:
        f = np.array([i if 2 * i < 6 else i - 6 for i in (i1, i2, i3)], dtype=float)
        g = np.linalg.norm((f + d) @ B)
        val, _ = integrate.quad(lambda r: special.erfc(mu * r), 0, np.inf, weight="sin", wvar=g)
        ref = 4 * math.pi / g * val
        assert abs(v[i3, i2, i1] - ref) <= 1e-8 * abs(ref)
    # g = 0: limit pi / mu^2 = 4 pi int r erfc(mu r) dr
    v0 = oracle_mod.kernel_grid(lat, grid, np.zeros(3), synth.KERNEL_HSE, mu)[0, 0, 0]
    val, _ = integrate.quad(lambda r: r * special.erfc(mu * r), 0, np.inf)
    assert abs(v0 - 4 * math.pi * val) <= 1e-8 * v0


def test_kernel_derivative_in_mu(oracle_mod):
    lat = synth.rhombohedral_lattice(9.56, 58.06)
    grid, d, mu, h = (8, 8, 8), np.array([0.125, 0.375, -0.375]), 0.106, 1e-5
    dv = oracle_mod.kernel_grid(lat, grid, d, 0, mu, which=1)
    fd = (oracle_mod.kernel_grid(lat, grid, d, 0, mu + h) -
          oracle_mod.kernel_grid(lat, grid, d, 0, mu - h)) / (2 * h)
    assert np.abs(dv - fd).max() <= 1e-6 * np.abs(dv).max()
    dv0 = oracle_mod.kernel_grid(lat, grid, np.zeros(3), 0, mu, which=1)[0, 0, 0]
    assert abs(dv0 - (-2 * math.pi / mu ** 3)) <= 1e-14 * abs(dv0)


def test_coulomb_kernel_drops_only_g0(oracle_mod):
    lat = synth.cubic_lattice(10.0)
    v = oracle_mod.kernel_grid(lat, (6, 6, 6), np.zeros(3), synth.KERNEL_COULOMB, 0.0)
    assert v[0, 0, 0] == 0.0
    assert abs(v[0, 0, 1] - 4 * math.pi / (2 * math.pi / 10.0) ** 2) <= 1e-14 * v[0, 0, 1]
    # screened kernel tends to Coulomb as mu -> 0 (g != 0)
    vs = oracle_mod.kernel_grid(lat, (6, 6, 6), np.zeros(3), synth.KERNEL_HSE, 1e-3)
    mask = v > 0
    assert np.abs(vs[mask] - v[mask]).max() <= 1e-12 * v[mask].max()


# ------------------------------------------------------------ one band pair

@pytest.mark.parametrize("shape", [(8, 6, 10), (12, 12, 12)])
def test_pair_potential_is_circular_convolution(oracle_mod, shape):
    """W(r_p) = sum_p' K(r_p - r_p') rho(r_p'), K(r) = (1/N) sum_G v(d+G) e^{iG.r}, all O(N^2)."""
    rng = np.random.default_rng(7)
    lat = synth.rhombohedral_lattice(6.0, 70.0)
    grid = (shape[2], shape[1], shape[0])
    d = np.array([0.5, 0.0, -0.25])
    u_j, u_a = rand_c(rng, shape), rand_c(rng, shape)
    W = oracle_mod.pair_potential(lat, grid, d, 0, 0.3, u_j, u_a)
    v = oracle_mod.kernel_grid(lat, grid, d, 0, 0.3)
    n3, n2, n1 = shape
    N = u_j.size
    K = direct_dft3(v, +1) / N                   # K on the grid, direct DFT
    rho = np.conj(u_j) * u_a
    i3, i2, i1 = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    idx = np.stack([i3.ravel(), i2.ravel(), i1.ravel()], 1)
    dif = (idx[:, None, :] - idx[None, :, :]) % np.array([n3, n2, n1])
    Kmat = K[dif[..., 0], dif[..., 1], dif[..., 2]]
    ref = (Kmat @ rho.ravel()).reshape(shape)
    assert np.abs(W - ref).max() <= 1e-12 * np.abs(ref).max()


# ------------------------------------------------------------ full operator

@pytest.mark.parametrize("make", [small_cubic, small_rhombo,
                                  lambda: small_cubic(kernel=synth.KERNEL_COULOMB),
                                  lambda: small_rhombo(kernel=synth.KERNEL_COULOMB)])
def test_apply_equals_coefficient_space_double_convolution(oracle_mod, make):
    wl = make()
    got = oracle_mod.apply(wl)
    ref = coeffspace.apply(wl)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_every_admissible_grid_gives_the_same_operator(oracle_mod):
    """Under the no-wrap-around reading every grid with N >= 4 n_max + 1 gives the same
    V_x c and E_x: the oracle on the tiny cell's 24^3 grid (n_max = 4, 4 n_max + 1 = 17)
    against 18^3 and 20^3, and a grid below the bound (16^3) that does alias."""
    wl = synth.tiny_cubic()
    assert int(wl.n_max().max()) == 4
    ref = oracle_mod.apply(wl)
    e_ref, _ = oracle_mod.energy_from_vx(wl, ref)
    for n in (18, 20):
        other = wl.replace(grid=(n,) * 3)
        vx = oracle_mod.apply(other)
        e, _ = oracle_mod.energy_from_vx(other, vx)
        assert np.abs(vx - ref).max() <= 1e-12 * np.abs(ref).max()
        assert abs(e - e_ref) <= 1e-12 * abs(e_ref)
    aliased = oracle_mod.apply(wl.replace(grid=(16,) * 3))
    assert np.abs(aliased - ref).max() > 1e-6 * np.abs(ref).max()


def test_anisotropic_grids_give_the_same_operator(oracle_mod):
    """Grids of different lengths per axis, each admissible on its own axis: a
    sheared cell elongated along a2 (n_max = (4, 6, 5)) on 17 x 25 x 21 (the
    smallest admissible), 24 x 32 x 24 and 18 x 27 x 24 gives the same V_x c as on
    32^3, and a grid aliasing along the long axis only (32 x 23 x 32) does not."""
    lat = np.array([[10.0, 0.0, 0.0], [1.5, 13.3, 0.0], [0.8, -1.1, 10.0]])
    wl = synth.make_workload("sheared", lat, (32, 32, 32), np.zeros((1, 3)), math.pi, 3, 4,
                             [1.0, 0.8, 0.5], 41)
    nm = wl.n_max()
    assert nm[1] > nm[0] and nm[1] > nm[2]
    ref = oracle_mod.apply(wl)
    assert tuple(int(v) for v in nm) == (4, 6, 5)
    for g in ((4 * nm[0] + 1, 4 * nm[1] + 1, 4 * nm[2] + 1), (24, 32, 24), (18, 27, 24)):
        vx = oracle_mod.apply(wl.replace(grid=tuple(int(v) for v in g)))
        assert np.abs(vx - ref).max() <= 1e-12 * np.abs(ref).max()
    aliased = oracle_mod.apply(wl.replace(grid=(32, 4 * int(nm[1]) - 1, 32)))
    assert np.abs(aliased - ref).max() > 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("make", [small_rhombo, synth.tiny_cubic])
def test_hermiticity(oracle_mod, make):
    wl = make()
    vx = oracle_mod.apply(wl)
    H = np.einsum("kag,kbg->kab", wl.c_tgt.conj(), vx)
    assert np.abs(H - np.conj(np.transpose(H, (0, 2, 1)))).max() <= 1e-13 * np.abs(H).max()


@pytest.mark.parametrize("make", [small_rhombo, synth.tiny_cubic])
def test_parseval_two_energy_forms(oracle_mod, make):
    wl = make()
    vx = oracle_mod.apply(wl)
    e_re, e_im = oracle_mod.energy_from_vx(wl, vx)
    e_ps = oracle_mod.pair_sum(wl, which=0)
    assert e_re < 0
    assert abs(e_re - e_ps) <= 1e-13 * abs(e_ps)
    assert abs(e_im) <= 1e-13 * abs(e_re)


# ------------------------------------------------------------- plane waves

def pw_closed_form(wl):
    """Exact V_x eigenvalues and E_x of single-plane-wave orbitals (Coulomb, G=0 dropped)."""
    m = wl.miller[0, :wl.npw[0]].astype(float)
    G = m @ coeffspace.reciprocal(wl.lattice)
    omega = abs(np.linalg.det(wl.lattice))
    d = G[:, None, :] - G[None, :, :]
    g2 = np.einsum("abi,abi->ab", d, d)
    np.fill_diagonal(g2, np.inf)
    lam = -(4 * math.pi / g2).sum(axis=1) / omega     # V_x c_a = lam_a c_a
    return lam, lam.sum()                               # E_x = (s/2) sum_a lam_a, s = 2


@pytest.mark.parametrize("shell", [2, 5])
def test_plane_wave_lattice_sum(oracle_mod, shell):
    wl = synth.plane_wave_cell(shell, grid=16)
    vx = oracle_mod.apply(wl)
    lam, ex = pw_closed_form(wl)
    ref = lam[:, None] * wl.c_tgt[0]
    assert np.abs(vx[0] - ref).max() <= 1e-12 * np.abs(lam).max()
    e, _ = oracle_mod.energy_from_vx(wl, vx)
    assert abs(e - ex) <= 1e-12 * abs(ex)


@pytest.mark.parametrize("shell", synth.PW_SHELLS)
def test_plane_wave_cells_approach_dirac_exchange(shell):
    """HEG exchange per electron -3 k_F / (4 pi), after the spherical q -> 0 correction."""
    wl = synth.plane_wave_cell(shell)
    _, ex = pw_closed_form(wl)
    omega = abs(np.linalg.det(wl.lattice))
    n_orb = wl.npw[0]
    n_e = 2 * n_orb
    kf = (3 * math.pi ** 2 * n_e / omega) ** (1 / 3)
    qc = (6 * math.pi ** 2 / omega) ** (1 / 3)
    corr = -n_orb * 16 * math.pi ** 2 * qc / (2 * math.pi) ** 3
    ratio = (ex + corr) / n_e / (-3 * kf / (4 * math.pi))
    assert abs(ratio - 1.0) <= 0.03


# -------------------------------------------------------------- invariances

def test_unitary_rotation_of_occupied_bands(oracle_mod):
    wl = small_rhombo()
    rng = np.random.default_rng(5)
    vx = oracle_mod.apply(wl)
    c_occ = wl.c_occ.copy()
    # rotate the two equally occupied bands (w = 1) among themselves, per k
    for k in range(wl.nk):
        q, _ = np.linalg.qr(rand_c(rng, (2, 2)))
        c_occ[k, :2] = q.T @ c_occ[k, :2]
    vx2 = oracle_mod.apply(wl, c_occ=c_occ)
    assert np.abs(vx2 - vx).max() <= 1e-12 * np.abs(vx).max()


def test_translation_invariance(oracle_mod):
    wl = small_rhombo()
    t = np.array([0.123, -0.377, 0.291])                # fractional translation
    c = wl.coeff.copy()
    for k in range(wl.nk):
        ph = np.exp(-2j * math.pi * (wl.miller[k] @ t))
        c[k] *= ph[None, :]
    wl2 = wl.replace(coeff=c)
    vx, vx2 = oracle_mod.apply(wl), oracle_mod.apply(wl2)
    e1, _ = oracle_mod.energy_from_vx(wl, vx)
    e2, _ = oracle_mod.energy_from_vx(wl2, vx2)
    assert abs(e1 - e2) <= 1e-12 * abs(e1)
    for k in range(wl.nk):
        ph = np.exp(-2j * math.pi * (wl.miller[k] @ t))
        assert np.abs(vx2[k] - vx[k] * ph[None, :]).max() <= 1e-12 * np.abs(vx).max()


# ---------------------------------------------------------------- gradients

def test_dmu_closed_form_matches_finite_difference(oracle_mod):
    wl = small_rhombo()
    h = 1e-4
    dmu = oracle_mod.pair_sum(wl, which=1)

    def cd(step):
        return (oracle_mod.pair_sum(wl, mu=wl.mu + step) -
                oracle_mod.pair_sum(wl, mu=wl.mu - step)) / (2 * step)
    # the O(h^2) term is 2 h^2 / mu^2 relative (~2e-6 at mu = 0.106): remove it by
    # Richardson extrapolation over steps h and 2h
    fd = (4 * cd(h) - cd(2 * h)) / 3
    assert abs(dmu - fd) <= 1e-8 * abs(dmu)


def test_dc_gradient_matches_finite_difference(oracle_mod):
    """dE/dc_ka* = (s w_ka / N_k) (V_x c)_ka; central FD along random directions."""
    wl = small_cubic(nb=4)
    c = wl.coeff.copy()
    vx = oracle_mod.apply(wl)
    grad = 2.0 * wl.w[:, :, None] / wl.nk * vx            # s = 2
    rng = np.random.default_rng(9)
    h = 1e-4
    for _ in range(16):
        dlt = rand_c(rng, c.shape)
        for k in range(wl.nk):
            dlt[k, :, wl.npw[k]:] = 0
        dlt /= np.linalg.norm(dlt)                      # unit direction
        ep = oracle_mod.energy(wl, c=c + h * dlt)
        em = oracle_mod.energy(wl, c=c - h * dlt)
        fd = (ep - em) / (2 * h)
        an = 2.0 * np.real(np.vdot(dlt, grad))
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-3 * np.abs(grad).max())


# ---------------------------------------------------- real orbitals at Gamma

def test_synthetic_real_orbitals_are_real_and_orthonormal():
    """The real-orbital generator: c(-G) = conj c(G), u(r) real, <c_a|c_b> = delta_ab."""
    wl = synth.real_tiny_cubic()
    n = int(wl.npw[0])
    c = wl.coeff[0, :, :n]
    assert np.abs(c.conj() @ c.T - np.eye(c.shape[0])).max() <= 1e-13
    neg = synth.minus_g_index(wl.miller[0, :n])
    assert np.array_equal(c[:, neg], c.conj())
    N = wl.grid[0]
    box = np.zeros((c.shape[0], N, N, N), dtype=np.complex128)
    m = wl.miller[0, :n] % N
    box[:, m[:, 0], m[:, 1], m[:, 2]] = c
    u = np.fft.ifftn(box, axes=(1, 2, 3))
    assert np.abs(u.imag).max() <= 1e-14 * np.abs(u.real).max()


@pytest.mark.parametrize("kernel", [synth.KERNEL_HSE, synth.KERNEL_COULOMB])
def test_exchange_of_real_orbitals_is_real(oracle_mod, kernel):
    """With real occupied orbitals and a real kernel even in G, V_x maps real
    functions to real functions: (V_x c)(-G) = conj (V_x c)(G) for real targets."""
    wl = synth.real_tiny_cubic(n_occ=3, n_tgt=4, kernel=kernel)
    vx = oracle_mod.apply(wl)[0]
    n = int(wl.npw[0])
    neg = synth.minus_g_index(wl.miller[0, :n])
    assert np.abs(vx[:, neg] - vx[:, :n].conj()).max() <= 1e-13 * np.abs(vx).max()
    # and every pair potential is real, W_aj = W_ja (the two bands of a packed
    # transform are its real and imaginary parts)
    m = wl.miller[0, :n]
    u = [oracle_mod.sphere_to_grid(wl.lattice, wl.grid, m, wl.coeff[0, b, :n]) for b in range(3)]
    d = np.zeros(3)
    W01 = oracle_mod.pair_potential(wl.lattice, wl.grid, d, kernel, wl.mu, u[1], u[0])
    W10 = oracle_mod.pair_potential(wl.lattice, wl.grid, d, kernel, wl.mu, u[0], u[1])
    assert np.abs(W01.imag).max() <= 1e-13 * np.abs(W01.real).max()
    assert np.abs(W01 - W10).max() <= 1e-13 * np.abs(W01).max()
    Wp = oracle_mod.pair_potential(wl.lattice, wl.grid, d, kernel, wl.mu, u[1] - 1j * u[2], u[0])
    W02 = oracle_mod.pair_potential(wl.lattice, wl.grid, d, kernel, wl.mu, u[2], u[0])
    assert np.abs(Wp - (W01 + 1j * W02)).max() <= 1e-13 * np.abs(Wp).max()
