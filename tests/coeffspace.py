"""Grid-free restatement of the exchange operator, used only to pin the oracle.

For band-limited orbitals on an alias-free grid the FFT pipeline of the paper's
exchange loops (Eq. 2 and the k, q, band, band loops around it) equals two
plain convolutions in coefficient space:

  rhohat_{ka,qj}(G') = Omega^{-1} sum_{G''} conj(c_qj(G'')) c_ka(G'' + G')
  (V_x c)_ka(G)      = -sum_{q,j} (w_qj / N_q) sum_{G'} c_qj(G - G') v(k - q + G') rhohat(G')

This module evaluates them by explicit shifts over dense Miller boxes, with no
FFT and no real-space grid, and with its own reciprocal lattice (numpy matrix
inverse) and kernel evaluation.
"""
import math

import numpy as np


def reciprocal(lattice):
    return 2.0 * math.pi * np.linalg.inv(np.asarray(lattice, dtype=np.float64)).T


def kernel_values(lattice, d, shifts, kernel, mu):
    """v(d + G') for integer shifts (n, 3); kernel 0 = screened, 1 = Coulomb (g=0 dropped)."""
    B = reciprocal(lattice)
    g = (shifts + np.asarray(d)[None, :]) @ B
    g2 = np.einsum("ij,ij->i", g, g)
    zero = np.all((shifts + np.asarray(d)[None, :]) == 0.0, axis=1)
    out = np.zeros_like(g2)
    nz = ~zero
    if kernel == 0:
        out[nz] = 4.0 * math.pi / g2[nz] * (1.0 - np.exp(-g2[nz] / (4.0 * mu * mu)))
        out[zero] = math.pi / (mu * mu)
    else:
        out[nz] = 4.0 * math.pi / g2[nz]
    return out


def _boxes(wl, c, n):
    """Dense boxes [nk][nb][2n+1]^3 (axis order m1, m2, m3) from sphere coefficients."""
    nk, nb, _ = c.shape
    L = 2 * n + 1
    box = np.zeros((nk, nb, L, L, L), dtype=np.complex128)
    for k in range(nk):
        m = wl.miller[k, :wl.npw[k]] + n
        box[k][:, m[:, 0], m[:, 1], m[:, 2]] = c[k, :, :wl.npw[k]]
    return box


def apply(wl, c_occ=None, w_occ=None, c_tgt=None):
    """(V_x c)[k][a][g] in sphere layout, by direct double convolution."""
    c_occ = wl.c_occ if c_occ is None else c_occ
    w_occ = wl.w_occ if w_occ is None else w_occ
    c_tgt = wl.c_tgt if c_tgt is None else c_tgt
    nk = wl.nk
    n = int(wl.n_max().max())
    L = 2 * n + 1
    omega = abs(np.linalg.det(wl.lattice))
    bo = _boxes(wl, c_occ, n)          # [q][j][L^3]
    bt = _boxes(wl, c_tgt, n)          # [k][a][L^3]
    # zero-padded copies so that every shift in [-2n, 2n] is a plain slice
    P = L + 4 * n
    po = np.zeros(bo.shape[:2] + (P, P, P), dtype=np.complex128)
    po[:, :, 2 * n:2 * n + L, 2 * n:2 * n + L, 2 * n:2 * n + L] = bo
    pt = np.zeros(bt.shape[:2] + (P, P, P), dtype=np.complex128)
    pt[:, :, 2 * n:2 * n + L, 2 * n:2 * n + L, 2 * n:2 * n + L] = bt
    rng = range(-2 * n, 2 * n + 1)
    shifts = np.array([[s1, s2, s3] for s1 in rng for s2 in rng for s3 in rng])
    out = np.zeros(bt.shape, dtype=np.complex128)
    for k in range(nk):
        for q in range(nk):
            d = wl.kfrac[k] - wl.kfrac[q]
            v = kernel_values(wl.lattice, d, shifts.astype(np.float64), wl.kernel, wl.mu)
            for si, s in enumerate(shifts):
                # box of c_ka shifted by s: element g of the slice is c_ka(g + s)
                sl = tuple(slice(2 * n + s[i], 2 * n + s[i] + L) for i in range(3))
                ca_s = pt[k][(slice(None),) + sl].reshape(bt.shape[1], -1)
                rho = (bo[q].reshape(bo.shape[1], -1).conj() @ ca_s.T) / omega   # [j][a]
                # c_qj(G - s): slice shifted by -s
                sl2 = tuple(slice(2 * n - s[i], 2 * n - s[i] + L) for i in range(3))
                cj_s = po[q][(slice(None),) + sl2].reshape(bo.shape[1], -1)   # [j][g]
                coef = -(w_occ[q][:, None] / nk) * v[si] * rho                # [j][a]
                out[k] += (coef.T @ cj_s).reshape(out[k].shape)
    res = np.zeros(c_tgt.shape, dtype=np.complex128)
    for k in range(nk):
        m = wl.miller[k, :wl.npw[k]] + n
        res[k, :, :wl.npw[k]] = out[k][:, m[:, 0], m[:, 1], m[:, 2]]
    return res
