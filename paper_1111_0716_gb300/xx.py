"""Python binding of libxx (ctypes): argument marshalling only.

Every step of the exchange computation runs in the CUDA library; this module
passes device pointers (torch tensors' ``data_ptr()``), sizes and the current
CUDA stream to the C entry points of ``include/xx.h`` under the same names.
There is no CPU fallback: if libxx.so is missing or no GPU is present, the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libxx.so")

XX_OK = 0
XX_FP32_MIXED = 0
XX_FP64 = 1
XX_KERNEL_HSE = 0
XX_KERNEL_COULOMB_G0_DROPPED = 1
SPIN = 2.0

STATUS = {
    0: "XX_OK", -1: "XX_ERR_INVALID_ARGUMENT", -2: "XX_ERR_UNSUPPORTED_GRID",
    -3: "XX_ERR_GRID_ALIASING", -4: "XX_ERR_OUT_OF_MEMORY", -5: "XX_ERR_CUDA",
    -6: "XX_ERR_DEVICE_FLAG", -7: "XX_ERR_TIMEOUT", -8: "XX_ERR_NO_DEVICE",
    -9: "XX_ERR_SIZE_LIMIT",
}
XX_NOALLOC_MAX_ROWS = 16384

# every symbol declared in include/xx.h
EXPORTS = ("xx_create", "xx_destroy", "xx_apply", "xx_apply_range", "xx_energy",
           "xx_energy_range", "xx_energy_from_vx", "xx_energy_from_vx_range",
           "xx_apply_backward", "xx_sync", "xx_set_batch", "xx_profile_enable",
           "xx_profile_read", "xx_plan_info", "xx_status_string", "xx_exact_grid",
           "xx_energy_from_vx_noalloc", "xx_run_many", "xx_apply_vjp", "xx_set_option",
           "xx_strain_derivative", "xx_measure_fma_rate", "xx_set_shard", "xx_shard_blocks",
           "xx_run_batched", "xx_exact_grid3")
XX_OPT_PAIR_SYMMETRY = 0
XX_OPT_REAL_GAMMA = 1
XX_OPT_TMA_PASS_B = 2
XX_OPT_STAGE_PASS_A = 3
XX_OPT_TEST_WAIT_EXPIRY = 4
XX_OPT_FUSED_VJP = 5
XX_OPT_ACC_LIMIT_MB = 6
XX_OPT_TABLE_CACHE = 7

PROF_CLASSES = ("pass_a", "pass_b", "pass_c", "sphere_to_grid", "grid_to_sphere",
                "kernel_table", "reduce", "pass_b_dmu")


class XXError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s failed: %s (%s)" % (where, STATUS.get(status, status),
                                                  xx_status_string(status)))


class xx_job(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("c_occ", ctypes.c_void_p), ("ld_occ", ctypes.c_int),
                ("w_occ", ctypes.c_void_p), ("n_occ", ctypes.c_int), ("c_tgt", ctypes.c_void_p),
                ("w_tgt", ctypes.c_void_p), ("n_tgt", ctypes.c_int), ("vx_out", ctypes.c_void_p),
                ("ex_out", ctypes.c_void_p)]


class xx_info(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int * 3), ("n_max", ctypes.c_int * 3),
                ("pruned", ctypes.c_int * 3), ("nk", ctypes.c_int), ("npw_max", ctypes.c_int),
                ("precision", ctypes.c_int), ("targets_per_batch", ctypes.c_int),
                ("occupied_per_batch", ctypes.c_int), ("omega", ctypes.c_double),
                ("workspace_bytes", ctypes.c_size_t), ("peak_workspace_bytes", ctypes.c_size_t),
                ("kernel_launches", ctypes.c_longlong), ("pairs_transformed", ctypes.c_longlong),
                ("q_per_batch", ctypes.c_int)]


_lib = None


def load(path: Optional[str] = None):
    """Load libxx.so (built in-tree by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libxx.so not built (%s): run __graft_entry__.build() first" % p)
    lib = ctypes.CDLL(p)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    lib.xx_create.argtypes = [ctypes.POINTER(P), P, P, I, P, P, I, P, I, D, I, S]
    lib.xx_destroy.argtypes = [P]
    lib.xx_apply.argtypes = [P, P, I, P, I, P, I, P, P]
    lib.xx_apply_range.argtypes = [P, I, I, P, I, P, I, P, I, P, P]
    lib.xx_energy.argtypes = [P, P, I, P, I, P, P, I, P, P, P]
    lib.xx_energy_range.argtypes = [P, I, I, P, I, P, I, P, P, I, P, P, P]
    lib.xx_energy_from_vx.argtypes = [P, P, P, I, P, P, P]
    lib.xx_energy_from_vx_range.argtypes = [P, I, I, P, P, I, P, P, P]
    lib.xx_apply_backward.argtypes = [P, P, P, I, P, D, P, P, P]
    lib.xx_sync.argtypes = [P, P, D]
    lib.xx_set_batch.argtypes = [P, I, I]
    lib.xx_plan_info.argtypes = [P, ctypes.POINTER(xx_info)]
    lib.xx_profile_enable.argtypes = [P, I]
    lib.xx_profile_read.argtypes = [P, P, P, I, I]
    lib.xx_energy_from_vx_noalloc.argtypes = [I, I, I, P, P, P, P, P, P]
    lib.xx_run_many.argtypes = [I, ctypes.POINTER(xx_job), P]
    lib.xx_run_batched.argtypes = [I, ctypes.POINTER(xx_job), P]
    lib.xx_apply_vjp.argtypes = [P, P, I, P, I, P, I, P, P, P, P]
    lib.xx_set_option.argtypes = [P, I, ctypes.c_longlong]
    lib.xx_strain_derivative.argtypes = [P, P, P, I, P, P, P]
    lib.xx_status_string.argtypes = [I]
    lib.xx_exact_grid.argtypes = [P, P]
    lib.xx_exact_grid3.argtypes = [P, P]
    lib.xx_measure_fma_rate.argtypes = [I, P, P]
    lib.xx_set_shard.argtypes = [P, I, I]
    lib.xx_shard_blocks.argtypes = [I, I, I, I, P]
    lib.xx_status_string.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("xx_status_string",):
            getattr(lib, name).restype = I
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != XX_OK:
        raise XXError(status, where)


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


_DTYPES = {"c128": "torch.complex128", "f64": "torch.float64", "i32": "torch.int32"}


def _dptr(t, name="tensor", kind=None, need=0, npw=None):
    """Device pointer of t (None passes as NULL).  The C entry points take plain
    pointers and cannot see sizes or types, so the binding checks them here: a
    contiguous CUDA tensor of the element type `kind` holding at least `need`
    elements; orbital arrays (npw given) must have the plan's padded basis
    length as their last dimension."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("%s: expected a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s: expected a contiguous tensor" % name)
    if kind is not None and str(t.dtype) != _DTYPES[kind]:
        raise ValueError("%s: expected %s, got %s" % (name, _DTYPES[kind], t.dtype))
    if t.numel() < need:
        raise ValueError("%s: holds %d elements, the call uses %d" % (name, t.numel(), need))
    if npw is not None and t.dim() >= 2 and t.shape[-1] != npw:
        raise ValueError("%s: last dimension %d, the plan's padded basis has %d"
                         % (name, t.shape[-1], npw))
    return ctypes.c_void_p(t.data_ptr())


def _dims(plan):
    """(nk, npw_max) of a plan, or None for a null or invalid handle (the C call
    then reports it)."""
    if plan is None or (isinstance(plan, ctypes.c_void_p) and not plan.value):
        return None
    info = xx_info()
    if load().xx_plan_info(plan, ctypes.byref(info)) != XX_OK:
        return None
    return int(info.nk), int(info.npw_max)


def _orbitals(plan, nk_used=None):
    """Helpers for one call: c(t, name, nb) checks a complex128 [nk][nb][npw_max]
    array, w(t, name, nb) a float64 [nk][nb] one, over nk_used k-points (all of
    the plan's by default); both pass everything when the plan is invalid."""
    d = _dims(plan)
    if d is None:
        return (lambda t, name, nb: _dptr(t, name)), (lambda t, name, nb: _dptr(t, name))
    nk, npw = d
    n = nk if nk_used is None else max(0, int(nk_used))
    return (lambda t, name, nb: _dptr(t, name, "c128", n * max(0, int(nb)) * npw, npw),
            lambda t, name, nb: _dptr(t, name, "f64", n * max(0, int(nb))))


def _ld(ld_occ, n_occ):
    return int(ld_occ) if int(ld_occ) > 0 else int(n_occ)


# ------------------------------------------------------- C entry points --

def xx_status_string(status: int) -> str:
    return load().xx_status_string(int(status)).decode()


def xx_create(lattice, grid, kfrac, npw, miller, kernel_type, mu, precision, workspace_cap=0):
    """Host arrays in, plan handle (c_void_p) out."""
    lat = np.ascontiguousarray(lattice, dtype=np.float64).reshape(9)
    g = np.ascontiguousarray(grid, dtype=np.int32).reshape(3)
    kf = np.ascontiguousarray(kfrac, dtype=np.float64).reshape(-1, 3)
    nk = kf.shape[0]
    npw_a = np.ascontiguousarray(npw, dtype=np.int32).reshape(nk)
    mil = np.ascontiguousarray(miller, dtype=np.int32).reshape(nk, -1, 3)
    plan = ctypes.c_void_p()
    _check(load().xx_create(ctypes.byref(plan), _np_ptr(lat), _np_ptr(g), nk, _np_ptr(kf),
                            _np_ptr(npw_a), mil.shape[1], _np_ptr(mil), int(kernel_type),
                            float(mu), int(precision), int(workspace_cap)), "xx_create")
    return plan


def xx_destroy(plan):
    _check(load().xx_destroy(plan), "xx_destroy")


def xx_apply(plan, c_occ, ld_occ, w_occ, n_occ, c_tgt, n_tgt, vx_out, stream=None):
    c, w = _orbitals(plan)
    _check(load().xx_apply(plan, c(c_occ, "c_occ", _ld(ld_occ, n_occ)), int(ld_occ),
                           w(w_occ, "w_occ", n_occ), int(n_occ), c(c_tgt, "c_tgt", n_tgt),
                           int(n_tgt), c(vx_out, "vx_out", n_tgt), _stream_ptr(stream)),
           "xx_apply")


def xx_apply_range(plan, k_first, k_count, c_occ, ld_occ, w_occ, n_occ, c_tgt, n_tgt, vx_out,
                   stream=None):
    c, w = _orbitals(plan)
    cr, _ = _orbitals(plan, k_count)
    _check(load().xx_apply_range(plan, int(k_first), int(k_count),
                                 c(c_occ, "c_occ", _ld(ld_occ, n_occ)), int(ld_occ),
                                 w(w_occ, "w_occ", n_occ), int(n_occ), cr(c_tgt, "c_tgt", n_tgt),
                                 int(n_tgt), cr(vx_out, "vx_out", n_tgt), _stream_ptr(stream)),
           "xx_apply_range")


def xx_energy_range(plan, k_first, k_count, c_occ, ld_occ, w_occ, n_occ, c_tgt, w_tgt, n_tgt,
                    vx_out, ex_out, stream=None):
    c, w = _orbitals(plan)
    cr, wr = _orbitals(plan, k_count)
    _check(load().xx_energy_range(plan, int(k_first), int(k_count),
                                  c(c_occ, "c_occ", _ld(ld_occ, n_occ)), int(ld_occ),
                                  w(w_occ, "w_occ", n_occ), int(n_occ), cr(c_tgt, "c_tgt", n_tgt),
                                  wr(w_tgt, "w_tgt", n_tgt), int(n_tgt),
                                  cr(vx_out, "vx_out", n_tgt), _dptr(ex_out, "ex_out", "f64", 2),
                                  _stream_ptr(stream)), "xx_energy_range")


def xx_energy_from_vx_range(plan, k_first, k_count, c_tgt, w_tgt, n_tgt, vx, ex_out, stream=None):
    cr, wr = _orbitals(plan, k_count)
    _check(load().xx_energy_from_vx_range(plan, int(k_first), int(k_count),
                                          cr(c_tgt, "c_tgt", n_tgt), wr(w_tgt, "w_tgt", n_tgt),
                                          int(n_tgt), cr(vx, "vx", n_tgt),
                                          _dptr(ex_out, "ex_out", "f64", 2), _stream_ptr(stream)),
           "xx_energy_from_vx_range")


def xx_energy(plan, c_occ, ld_occ, w_occ, n_occ, c_tgt, w_tgt, n_tgt, vx_out, ex_out, stream=None):
    c, w = _orbitals(plan)
    _check(load().xx_energy(plan, c(c_occ, "c_occ", _ld(ld_occ, n_occ)), int(ld_occ),
                            w(w_occ, "w_occ", n_occ), int(n_occ), c(c_tgt, "c_tgt", n_tgt),
                            w(w_tgt, "w_tgt", n_tgt), int(n_tgt), c(vx_out, "vx_out", n_tgt),
                            _dptr(ex_out, "ex_out", "f64", 2), _stream_ptr(stream)), "xx_energy")


def xx_energy_from_vx_noalloc(nk, n_tgt, npw_max, npw, c_tgt, w_tgt, vx, ex_out, stream=None):
    """E_x reduction without a plan or any device allocation (fixed device scratch)."""
    nk, n_tgt, npw_max = int(nk), int(n_tgt), int(npw_max)
    rows = max(0, nk) * max(0, n_tgt)
    _check(load().xx_energy_from_vx_noalloc(
        nk, n_tgt, npw_max, _dptr(npw, "npw", "i32", max(0, nk)),
        _dptr(c_tgt, "c_tgt", "c128", rows * max(0, npw_max)),
        _dptr(w_tgt, "w_tgt", "f64", rows), _dptr(vx, "vx", "c128", rows * max(0, npw_max)),
        _dptr(ex_out, "ex_out", "f64", 2), _stream_ptr(stream)), "xx_energy_from_vx_noalloc")


def xx_energy_from_vx(plan, c_tgt, w_tgt, n_tgt, vx, ex_out, stream=None):
    c, w = _orbitals(plan)
    _check(load().xx_energy_from_vx(plan, c(c_tgt, "c_tgt", n_tgt), w(w_tgt, "w_tgt", n_tgt),
                                    int(n_tgt), c(vx, "vx", n_tgt),
                                    _dptr(ex_out, "ex_out", "f64", 2), _stream_ptr(stream)),
           "xx_energy_from_vx")


def xx_apply_backward(plan, c, w, n_b, vx, grad_ex, dc_out, dmu_out, stream=None):
    co, wo = _orbitals(plan)
    _check(load().xx_apply_backward(plan, co(c, "c", n_b), wo(w, "w", n_b), int(n_b),
                                    co(vx, "vx", n_b), float(grad_ex), co(dc_out, "dc_out", n_b),
                                    _dptr(dmu_out, "dmu_out", "f64", 1), _stream_ptr(stream)),
           "xx_apply_backward")


def xx_apply_vjp(plan, c_occ, ld_occ, w_occ, n_occ, c_tgt, n_tgt, ybar, grad_tgt_out,
                 grad_occ_out, stream=None):
    c, w = _orbitals(plan)
    _check(load().xx_apply_vjp(plan, c(c_occ, "c_occ", _ld(ld_occ, n_occ)), int(ld_occ),
                               w(w_occ, "w_occ", n_occ), int(n_occ), c(c_tgt, "c_tgt", n_tgt),
                               int(n_tgt), c(ybar, "ybar", n_tgt),
                               c(grad_tgt_out, "grad_tgt_out", n_tgt),
                               c(grad_occ_out, "grad_occ_out", n_occ), _stream_ptr(stream)),
           "xx_apply_vjp")


def _job_array(jobs):
    arr = (xx_job * len(jobs))()
    for i, j in enumerate(jobs):
        n_occ = j["w_occ"].shape[1]
        ld = j.get("ld_occ", j["c_occ"].shape[1])
        n_tgt = j["c_tgt"].shape[1]
        c, w = _orbitals(j["plan"].handle)
        arr[i].plan = j["plan"].handle
        arr[i].c_occ = c(j["c_occ"], "c_occ", _ld(ld, n_occ))
        arr[i].ld_occ = int(ld)
        arr[i].w_occ = w(j["w_occ"], "w_occ", n_occ)
        arr[i].n_occ = int(n_occ)
        arr[i].c_tgt = c(j["c_tgt"], "c_tgt", n_tgt)
        arr[i].w_tgt = w(j.get("w_tgt"), "w_tgt", n_tgt)
        arr[i].n_tgt = int(n_tgt)
        arr[i].vx_out = c(j["vx_out"], "vx_out", n_tgt)
        arr[i].ex_out = _dptr(j.get("ex_out"), "ex_out", "f64", 2)
    return arr


def xx_run_many(jobs, stream=None):
    """jobs: list of dicts with keys plan (Plan), c_occ, w_occ, c_tgt, w_tgt, vx_out, ex_out
    (ex_out/w_tgt optional) and optional ld_occ; the occupied set is the leading bands when
    c_occ is c_tgt."""
    _check(load().xx_run_many(len(jobs), _job_array(jobs), _stream_ptr(stream)), "xx_run_many")


def xx_run_batched(jobs, stream=None):
    """Gamma-only jobs (same keys as xx_run_many) with one launch per band-pair pass."""
    _check(load().xx_run_batched(len(jobs), _job_array(jobs), _stream_ptr(stream)),
           "xx_run_batched")


def xx_sync(plan, stream=None, timeout_s: float = 0.0):
    _check(load().xx_sync(plan, _stream_ptr(stream), float(timeout_s)), "xx_sync")


def xx_strain_derivative(plan, c, w, n_b, dex_deps, ex_out=None, stream=None):
    co, wo = _orbitals(plan)
    _check(load().xx_strain_derivative(plan, co(c, "c", n_b), wo(w, "w", n_b), int(n_b),
                                       _dptr(dex_deps, "dex_deps", "f64", 9),
                                       _dptr(ex_out, "ex_out", "f64", 1), _stream_ptr(stream)),
           "xx_strain_derivative")


def xx_set_option(plan, option: int, value: int):
    _check(load().xx_set_option(plan, int(option), int(value)), "xx_set_option")


def xx_set_batch(plan, targets_per_batch: int, occupied_per_batch: int):
    _check(load().xx_set_batch(plan, int(targets_per_batch), int(occupied_per_batch)),
           "xx_set_batch")


def xx_profile_enable(plan, enable: bool):
    _check(load().xx_profile_enable(plan, 1 if enable else 0), "xx_profile_enable")


def xx_profile_read(plan, reset: bool = True) -> dict:
    """{class: (ms, launch groups)} of the per-kernel-class event timing."""
    n = len(PROF_CLASSES)
    ms = np.zeros(n, dtype=np.float64)
    cnt = np.zeros(n, dtype=np.int64)
    _check(load().xx_profile_read(plan, _np_ptr(ms), _np_ptr(cnt), n, 1 if reset else 0),
           "xx_profile_read")
    return {c: (float(ms[i]), int(cnt[i])) for i, c in enumerate(PROF_CLASSES)}


def xx_exact_grid(n_max) -> int:
    """Smallest supported cubic FFT length N >= 4 n_max + 1 (the operator is exact there)."""
    nm = np.ascontiguousarray(np.asarray(n_max, dtype=np.int32).reshape(3))
    out = np.zeros(1, dtype=np.int32)
    _check(load().xx_exact_grid(_np_ptr(nm), _np_ptr(out)), "xx_exact_grid")
    return int(out[0])


def xx_set_shard(plan, shard: int, n_shards: int):
    _check(load().xx_set_shard(plan, int(shard), int(n_shards)), "xx_set_shard")


def xx_shard_blocks(nk: int, n_occ: int, n_tgt: int, n_shards: int) -> np.ndarray:
    """Owner shard of each k-point block {k <= q} (upper triangle, row-major)."""
    out = np.zeros(nk * (nk + 1) // 2, dtype=np.int32)
    _check(load().xx_shard_blocks(int(nk), int(n_occ), int(n_tgt), int(n_shards), _np_ptr(out)),
           "xx_shard_blocks")
    return out


def xx_measure_fma_rate(precision: int, stream=None) -> float:
    """Measured FMA rate (TFLOP/s) of the current device in FP32 or FP64 (blocking)."""
    out = np.zeros(1, dtype=np.float64)
    _check(load().xx_measure_fma_rate(int(precision), _np_ptr(out), _stream_ptr(stream)),
           "xx_measure_fma_rate")
    return float(out[0])


def xx_exact_grid3(n_max) -> tuple:
    """Fewest-point supported grid (two lengths equal) with N_i >= 4 n_max,i + 1 per axis."""
    nm = np.ascontiguousarray(np.asarray(n_max, dtype=np.int32).reshape(3))
    out = np.zeros(3, dtype=np.int32)
    _check(load().xx_exact_grid3(_np_ptr(nm), _np_ptr(out)), "xx_exact_grid3")
    return tuple(int(v) for v in out)


def xx_plan_info(plan) -> dict:
    info = xx_info()
    _check(load().xx_plan_info(plan, ctypes.byref(info)), "xx_plan_info")
    return {f: (list(getattr(info, f)) if isinstance(getattr(info, f), ctypes.Array)
                else getattr(info, f)) for f, _ in xx_info._fields_}


# ------------------------------------------------------------ high level --

class Plan:
    """Owns an xx_plan for one cell / grid / k-mesh / basis (and kernel, precision)."""

    def __init__(self, lattice, grid, kfrac, npw, miller, kernel=XX_KERNEL_HSE, mu=0.106,
                 precision=XX_FP32_MIXED, workspace_cap=0):
        self.handle = xx_create(lattice, grid, kfrac, npw, miller, kernel, mu, precision,
                                workspace_cap)
        self.nk = int(np.asarray(kfrac).reshape(-1, 3).shape[0])
        self.npw_max = int(np.asarray(miller).reshape(self.nk, -1, 3).shape[1])
        self.kernel = kernel
        self.mu = float(mu)
        self.precision = precision

    @classmethod
    def from_workload(cls, wl, precision=XX_FP32_MIXED, mu=None, workspace_cap=0):
        return cls(wl.lattice, wl.grid, wl.kfrac, wl.npw, wl.miller, kernel=wl.kernel,
                   mu=wl.mu if mu is None else mu, precision=precision,
                   workspace_cap=workspace_cap)

    def close(self):
        if getattr(self, "handle", None) is not None:
            xx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        return xx_plan_info(self.handle)

    def profile(self, enable: bool = True):
        xx_profile_enable(self.handle, enable)

    def profile_read(self, reset: bool = True) -> dict:
        return xx_profile_read(self.handle, reset)

    def set_shard(self, shard: int, n_shards: int):
        """Compute only the k-point blocks assigned to shard `shard` of `n_shards`."""
        xx_set_shard(self.handle, shard, n_shards)

    def set_pair_symmetry(self, enable: bool):
        xx_set_option(self.handle, XX_OPT_PAIR_SYMMETRY, 1 if enable else 0)

    def set_tma_pass_b(self, mode: int):
        """0: one-row-per-block pass B; 1: automatic (default); 2: tensor-copy kernel."""
        xx_set_option(self.handle, XX_OPT_TMA_PASS_B, int(mode))

    def set_table_cache(self, enable: bool):
        """Keep the kernel tables of every (k, q) (default) or build them per batch."""
        xx_set_option(self.handle, XX_OPT_TABLE_CACHE, 1 if enable else 0)

    def set_stage_pass_a(self, mode: int):
        """0: two CTAs per SM with global loads; 1: automatic (default); 2: staged."""
        xx_set_option(self.handle, XX_OPT_STAGE_PASS_A, int(mode))

    def set_real_gamma(self, enable: bool):
        """Declare the orbitals of later calls real in real space (Gamma-only plans)."""
        xx_set_option(self.handle, XX_OPT_REAL_GAMMA, 1 if enable else 0)

    def set_batch(self, targets: int, occupied: int):
        xx_set_batch(self.handle, targets, occupied)

    def apply(self, c_occ, w_occ, c_tgt, vx_out=None, stream=None):
        """V_x c_tgt.  c_* complex128 CUDA tensors [nk][nb][npw_max]; w_occ float64 [nk][n_occ]."""
        import torch
        n_occ = c_occ.shape[1]
        n_tgt = c_tgt.shape[1]
        if vx_out is None:
            vx_out = torch.empty_like(c_tgt)
        xx_apply(self.handle, c_occ, n_occ, w_occ, n_occ, c_tgt, n_tgt, vx_out, stream)
        return vx_out

    def apply_shared(self, c, w_occ, n_occ, vx_out=None, stream=None):
        """V_x c for all bands of c, occupied set = the first n_occ bands of c (grids shared)."""
        import torch
        n_tgt = c.shape[1]
        if vx_out is None:
            vx_out = torch.empty_like(c)
        xx_apply(self.handle, c, n_tgt, w_occ, n_occ, c, n_tgt, vx_out, stream)
        return vx_out

    def apply_range(self, k_first, k_count, c_occ, w_occ, c_tgt, vx_out=None, stream=None):
        """V_x c_tgt for target k-points k_first..k_first+k_count-1 (c_tgt holds only those)."""
        import torch
        n_occ = c_occ.shape[1]
        if vx_out is None:
            vx_out = torch.empty_like(c_tgt)
        xx_apply_range(self.handle, k_first, k_count, c_occ, n_occ, w_occ, n_occ, c_tgt,
                       c_tgt.shape[1], vx_out, stream)
        return vx_out

    def energy_range(self, k_first, k_count, c_occ, w_occ, c_tgt, w_tgt, vx_out=None,
                     ex_out=None, stream=None):
        import torch
        if vx_out is None:
            vx_out = torch.empty_like(c_tgt)
        if ex_out is None:
            ex_out = torch.empty(2, dtype=torch.float64, device=c_tgt.device)
        n_occ = c_occ.shape[1]
        xx_energy_range(self.handle, k_first, k_count, c_occ, n_occ, w_occ, n_occ, c_tgt, w_tgt,
                        c_tgt.shape[1], vx_out, ex_out, stream)
        return ex_out, vx_out

    def energy(self, c_occ, w_occ, c_tgt, w_tgt, vx_out=None, ex_out=None, stream=None,
               shared=False):
        """(E_x as a device float64[2] (Re, Im), V_x c_tgt)."""
        import torch
        n_tgt = c_tgt.shape[1]
        n_occ = w_occ.shape[1]
        if vx_out is None:
            vx_out = torch.empty_like(c_tgt)
        if ex_out is None:
            ex_out = torch.empty(2, dtype=torch.float64, device=c_tgt.device)
        ld = n_tgt if shared else n_occ
        xx_energy(self.handle, c_tgt if shared else c_occ, ld, w_occ, n_occ, c_tgt, w_tgt, n_tgt,
                  vx_out, ex_out, stream)
        return ex_out, vx_out

    def backward(self, c, w, grad_ex=1.0, vx=None, want_dc=True, want_dmu=True, stream=None):
        import torch
        n_b = c.shape[1]
        dc = torch.empty_like(c) if want_dc else None
        dmu = torch.empty(1, dtype=torch.float64, device=c.device) if want_dmu else None
        xx_apply_backward(self.handle, c, w, n_b, vx, grad_ex, dc, dmu, stream)
        return dc, dmu

    def vjp(self, c_occ, w_occ, c_tgt, ybar, want_tgt=True, want_occ=True, stream=None):
        """(dL/dc_tgt*, dL/dc_occ*) for the cotangent ybar = dL/d(V_x c_tgt)*."""
        import torch
        gt = torch.empty_like(c_tgt) if want_tgt else None
        go = torch.empty_like(c_occ) if want_occ else None
        n_occ = c_occ.shape[1]
        xx_apply_vjp(self.handle, c_occ, n_occ, w_occ, n_occ, c_tgt, c_tgt.shape[1], ybar, gt, go,
                     stream)
        return gt, go

    def strain_derivative(self, c, w, stream=None):
        """(dE_x/deps as a device 3x3 float64, E_x) for orbitals c that are occupied and targets."""
        import torch
        d = torch.empty(9, dtype=torch.float64, device=c.device)
        e = torch.empty(1, dtype=torch.float64, device=c.device)
        xx_strain_derivative(self.handle, c, w, c.shape[1], d, e, stream)
        return d.reshape(3, 3), e

    def sync(self, timeout_s: float = 0.0, stream=None):
        xx_sync(self.handle, stream, timeout_s)


def _exchange_function():
    import torch

    class ExchangeEnergy(torch.autograd.Function):
        """E_x[c] with c both occupied and target (the usual self-consistent case).

        forward(c, w, mu, plan) -> E_x (float64 scalar).  ``mu`` is a float64
        tensor equal to the plan's screening parameter; its gradient is
        dE_x/dmu.  The complex gradient follows torch's convention
        (2 dL/dc*): 2 grad (s w / N_k) V_x c.  The backward reuses V_x c saved by
        the forward and recomputes codensities for dE_x/dmu (no pair grids are
        stored).
        """

        @staticmethod
        def forward(ctx, c, w, mu, plan):
            c = c.contiguous()
            w = w.contiguous()
            ex, vx = plan.energy(c, w, c, w, shared=True)
            ctx.plan = plan
            ctx.save_for_backward(c, w, vx)
            return ex[0]

        @staticmethod
        def backward(ctx, grad_out):
            c, w, vx = ctx.saved_tensors
            plan = ctx.plan
            g = float(grad_out.item())
            want_dc = ctx.needs_input_grad[0]
            want_dmu = ctx.needs_input_grad[2] and plan.kernel == XX_KERNEL_HSE
            dc, dmu = plan.backward(c, w, grad_ex=g, vx=vx, want_dc=want_dc, want_dmu=want_dmu)
            gc = 2.0 * dc if dc is not None else None
            gmu = dmu.reshape(()) if dmu is not None else None
            return gc, None, gmu, None

    return ExchangeEnergy


def _apply_function():
    import torch

    class ExchangeApply(torch.autograd.Function):
        """y = V_x[c_occ] c_tgt with gradients for both orbital sets.

        forward(c_occ, w_occ, c_tgt, plan) -> y.  torch's complex gradients are
        2 dL/dz*: backward passes grad_y / 2 as the Wirtinger cotangent to
        xx_apply_vjp and doubles the results.  Occupations get no gradient.
        """

        @staticmethod
        def forward(ctx, c_occ, w_occ, c_tgt, plan):
            c_occ, w_occ, c_tgt = c_occ.contiguous(), w_occ.contiguous(), c_tgt.contiguous()
            ctx.plan = plan
            ctx.save_for_backward(c_occ, w_occ, c_tgt)
            return plan.apply(c_occ, w_occ, c_tgt)

        @staticmethod
        def backward(ctx, grad_y):
            c_occ, w_occ, c_tgt = ctx.saved_tensors
            ybar = (0.5 * grad_y).contiguous()
            gt, go = ctx.plan.vjp(c_occ, w_occ, c_tgt, ybar, want_tgt=ctx.needs_input_grad[2],
                                  want_occ=ctx.needs_input_grad[0])
            return (2.0 * go if go is not None else None, None,
                    2.0 * gt if gt is not None else None, None)

    return ExchangeApply


_EXA = None


def exchange_apply(c_occ, w_occ, c_tgt, plan):
    """Differentiable V_x[c_occ] c_tgt (see ExchangeApply)."""
    global _EXA
    if _EXA is None:
        _EXA = _apply_function()
    return _EXA.apply(c_occ, w_occ, c_tgt, plan)


_EXF = None


def exchange_energy(c, w, mu, plan):
    """Differentiable E_x[c] (see ExchangeEnergy)."""
    global _EXF
    if _EXF is None:
        _EXF = _exchange_function()
    return _EXF.apply(c, w, mu, plan)
