"""Python wrapper over the FP64 CPU oracle (``xx_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg call this module; the product path never does.  It is independent
of the CUDA library: it neither imports the package's binding nor shares any of
its code.  Every function follows the steps of the paper's exchange loops
(Hutchinson & Widom, Sec. "Our Implementation", Eq. 2): see ``xx_oracle.c``.
"""
from __future__ import annotations

import ctypes
import fcntl
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xx_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP); returns the library path."""
    with open(_LIB + ".lock", "w") as fh:
        fcntl.flock(fh, fcntl.LOCK_EX)
        try:
            return _build_oracle(force)
        finally:
            fcntl.flock(fh, fcntl.LOCK_UN)


def _build_oracle(force: bool) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    """The loaded oracle library.  XX_ORACLE_LIB names another compiled copy of
    ``xx_oracle.c`` to load instead (the tests use it to check that the pins
    reject deliberately broken copies); otherwise the source is built here."""
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(os.environ.get("XX_ORACLE_LIB") or build_oracle())
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        _lib.oracle_fft3d.argtypes = [P, I, I, I, I]
        _lib.oracle_cell_volume.argtypes = [P]
        _lib.oracle_cell_volume.restype = D
        _lib.oracle_kernel_grid.argtypes = [P, P, P, I, D, I, P]
        _lib.oracle_sphere_to_grid.argtypes = [P, P, I, P, P, P]
        _lib.oracle_grid_to_sphere.argtypes = [P, P, I, P, P, P]
        _lib.oracle_pair_potential.argtypes = [P, P, P, I, D, P, P, P]
        _lib.oracle_apply.argtypes = [P, P, I, P, P, I, P, I, D, P, P, I, P, I, P, I, P]
        _lib.oracle_energy_from_vx.argtypes = [I, P, I, P, P, I, P, P]
        _lib.oracle_energy_from_vx.restype = D
        _lib.oracle_pair_sum.argtypes = [P, P, I, P, P, I, P, I, D, I, P, P, I, P, P, I]
        _lib.oracle_pair_sum.restype = D
        _lib.oracle_num_threads.restype = I
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def fft3d(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised 3D DFT of x[i3][i2][i1]; sign -1 forward, +1 inverse."""
    y = _c(x, np.complex128).copy()
    n3, n2, n1 = y.shape
    lib().oracle_fft3d(_p(y), n1, n2, n3, int(sign))
    return y


def cell_volume(lattice) -> float:
    return float(lib().oracle_cell_volume(_p(_c(lattice, np.float64))))


def kernel_grid(lattice, grid, d, kernel, mu, which=0) -> np.ndarray:
    """v(d + G) (which=0) or dv/dmu (which=1) on the FFT grid, shape (N3, N2, N1)."""
    g = _c(grid, np.int32)
    out = np.zeros((g[2], g[1], g[0]), dtype=np.float64)
    lib().oracle_kernel_grid(_p(_c(lattice, np.float64)), _p(g), _p(_c(d, np.float64)),
                             int(kernel), float(mu), int(which), _p(out))
    return out


def sphere_to_grid(lattice, grid, miller, c) -> np.ndarray:
    g = _c(grid, np.int32)
    m = _c(miller, np.int32)
    u = np.zeros((g[2], g[1], g[0]), dtype=np.complex128)
    lib().oracle_sphere_to_grid(_p(_c(lattice, np.float64)), _p(g), m.shape[0], _p(m),
                                _p(_c(c, np.complex128)), _p(u))
    return u


def grid_to_sphere(lattice, grid, miller, f) -> np.ndarray:
    g = _c(grid, np.int32)
    m = _c(miller, np.int32)
    ff = _c(f, np.complex128).copy()
    c = np.zeros(m.shape[0], dtype=np.complex128)
    lib().oracle_grid_to_sphere(_p(_c(lattice, np.float64)), _p(g), m.shape[0], _p(m),
                                _p(ff), _p(c))
    return c


def pair_potential(lattice, grid, d, kernel, mu, u_j, u_a) -> np.ndarray:
    g = _c(grid, np.int32)
    W = np.zeros((g[2], g[1], g[0]), dtype=np.complex128)
    lib().oracle_pair_potential(_p(_c(lattice, np.float64)), _p(g), _p(_c(d, np.float64)),
                                int(kernel), float(mu), _p(_c(u_j, np.complex128)),
                                _p(_c(u_a, np.complex128)), _p(W))
    return W


def apply(wl, sel=None, c_occ=None, w_occ=None, c_tgt=None, mu=None) -> np.ndarray:
    """V_x c for a Workload.  sel: list of (k, a) or None (all, k-major).

    Returns (n_sel, npw_max) complex128, or (nk, n_tgt, npw_max) when sel is None.
    """
    c_occ = _c(wl.c_occ if c_occ is None else c_occ, np.complex128)
    w_occ = _c(wl.w_occ if w_occ is None else w_occ, np.float64)
    c_tgt = _c(wl.c_tgt if c_tgt is None else c_tgt, np.complex128)
    nk, n_occ, npw_max = c_occ.shape
    n_tgt = c_tgt.shape[1]
    g = _c(wl.grid, np.int32)
    if sel is None:
        n_sel, sp = nk * n_tgt, None
    else:
        s = _c(np.asarray(sel).reshape(-1, 2), np.int32)
        n_sel, sp = s.shape[0], s
    out = np.zeros((n_sel, npw_max), dtype=np.complex128)
    lib().oracle_apply(_p(_c(wl.lattice, np.float64)), _p(g), nk, _p(_c(wl.kfrac, np.float64)),
                       _p(_c(wl.npw, np.int32)), npw_max, _p(_c(wl.miller, np.int32)),
                       int(wl.kernel), float(wl.mu if mu is None else mu), _p(c_occ), _p(w_occ),
                       n_occ, _p(c_tgt), n_tgt, None if sp is None else _p(sp), n_sel, _p(out))
    if sel is None:
        return out.reshape(nk, n_tgt, npw_max)
    return out


def energy_from_vx(wl, vx, c_tgt=None, w_tgt=None):
    """(Re, Im) of E_x = (s/2)(1/N_k) sum_ka w_ka <c_ka|V_x c_ka>."""
    c_tgt = _c(wl.c_tgt if c_tgt is None else c_tgt, np.complex128)
    w_tgt = _c(wl.w_tgt if w_tgt is None else w_tgt, np.float64)
    vx = _c(vx, np.complex128)
    nk, n_tgt, npw_max = c_tgt.shape
    im = np.zeros(1)
    re = lib().oracle_energy_from_vx(nk, _p(_c(wl.npw, np.int32)), npw_max, _p(c_tgt),
                                     _p(w_tgt), n_tgt, _p(vx), _p(im))
    return float(re), float(im[0])


def pair_sum(wl, which=0, c_occ=None, w_occ=None, c_tgt=None, w_tgt=None, mu=None) -> float:
    """-(s/2)(Omega/(N_k N_q)) sum w_ka w_qj sum_G K |rhohat|^2; K = v or dv/dmu."""
    c_occ = _c(wl.c_occ if c_occ is None else c_occ, np.complex128)
    w_occ = _c(wl.w_occ if w_occ is None else w_occ, np.float64)
    c_tgt = _c(wl.c_tgt if c_tgt is None else c_tgt, np.complex128)
    w_tgt = _c(wl.w_tgt if w_tgt is None else w_tgt, np.float64)
    nk, n_occ, npw_max = c_occ.shape
    return float(lib().oracle_pair_sum(
        _p(_c(wl.lattice, np.float64)), _p(_c(wl.grid, np.int32)), nk,
        _p(_c(wl.kfrac, np.float64)), _p(_c(wl.npw, np.int32)), npw_max,
        _p(_c(wl.miller, np.int32)), int(wl.kernel), float(wl.mu if mu is None else mu),
        int(which), _p(c_occ), _p(w_occ), n_occ, _p(c_tgt), _p(w_tgt), c_tgt.shape[1]))


def energy(wl, mu=None, c=None):
    """E_x of a workload whose targets are its occupied bands (full apply + reduction)."""
    c_all = wl.c_tgt if c is None else c
    vx = apply(wl, c_occ=c_all[:, :wl.n_occ], c_tgt=c_all, mu=mu)
    return energy_from_vx(wl, vx, c_tgt=c_all)[0]
