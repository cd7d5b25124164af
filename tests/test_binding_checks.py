"""The Python binding's argument checks, on CPU with a stand-in library.

The C entry points take plain pointers, so they cannot see a tensor's element
type or size: a complex64 array, or one with fewer bands than the call names,
would be read out of bounds on the GPU.  The binding checks type, size and the
padded basis length against the plan before it calls the library.  These tests
replace the library with a recorder and the tensors with stand-ins that only
carry the attributes the binding reads, so they need no GPU.
"""
import ctypes
import types

import pytest

torch = pytest.importorskip("torch")

from paper_1111_0716_gb300 import xx  # noqa: E402

NK, NPW = 4, 37
PLAN = ctypes.c_void_p(0x1000)


class T:
    """Stand-in for a CUDA tensor: shape, dtype, contiguity, a fake address."""

    def __init__(self, *shape, dtype=torch.complex128, cuda=True, contiguous=True):
        self.shape = tuple(shape)
        self.dtype = dtype
        self.is_cuda = cuda
        self._contiguous = contiguous

    def numel(self):
        n = 1
        for s in self.shape:
            n *= s
        return n

    def dim(self):
        return len(self.shape)

    def is_contiguous(self):
        return self._contiguous

    def data_ptr(self):
        return 0x2000


class Recorder:
    """Library stand-in: records entry-point calls, knows one plan (NK k-points,
    NPW padded basis)."""

    def __init__(self):
        self.calls = []

    def xx_plan_info(self, plan, ref):
        if plan is None or not getattr(plan, "value", plan):
            return -1
        ref._obj.nk = NK
        ref._obj.npw_max = NPW
        return 0

    def xx_status_string(self, status):
        return b"status"

    def __getattr__(self, name):
        def call(*args):
            self.calls.append(name)
            return 0
        return call


@pytest.fixture()
def lib(monkeypatch):
    rec = Recorder()
    monkeypatch.setattr(xx, "_lib", rec)
    return rec


S = types.SimpleNamespace(cuda_stream=0)


def c(nb, nk=NK, npw=NPW, **kw):
    return T(nk, nb, npw, **kw)


def w(nb, nk=NK, dtype=torch.float64, **kw):
    return T(nk, nb, dtype=dtype, **kw)


def f64(n):
    return T(n, dtype=torch.float64)


def test_valid_calls_reach_the_library(lib):
    ct, wt, vx = c(6), w(6), c(6)
    xx.xx_apply(PLAN, ct, 6, w(4), 4, ct, 6, vx, S)               # occupied = leading targets
    xx.xx_apply(PLAN, c(4), 4, w(4), 4, ct, 6, vx, S)             # separate occupied set
    xx.xx_apply(PLAN, c(4), 0, w(4), 4, ct, 6, vx, S)             # ld_occ 0 means n_occ
    xx.xx_apply(PLAN, ct, 0, w(4), 0, ct, 6, vx, S)               # no occupied bands
    xx.xx_apply(PLAN, ct, 0, w(4), 4, ct, 0, vx, S)               # no targets
    xx.xx_energy(PLAN, ct, 6, w(4), 4, ct, wt, 6, vx, f64(2), S)
    xx.xx_apply_range(PLAN, 1, 2, c(4), 4, w(4), 4, c(6, nk=2), 6, c(6, nk=2), S)
    xx.xx_energy_range(PLAN, 3, 1, c(4), 4, w(4), 4, c(6, nk=1), w(6, nk=1), 6, c(6, nk=1),
                       f64(2), S)
    xx.xx_energy_from_vx(PLAN, ct, wt, 6, vx, f64(2), S)
    xx.xx_energy_from_vx_range(PLAN, 0, 2, c(6, nk=2), w(6, nk=2), 6, c(6, nk=2), f64(2), S)
    xx.xx_apply_backward(PLAN, ct, wt, 6, None, 1.0, None, f64(1), S)
    xx.xx_apply_backward(PLAN, ct, wt, 6, vx, 1.0, c(6), None, S)
    xx.xx_apply_vjp(PLAN, ct, 6, w(4), 4, ct, 6, c(6), c(6), c(4), S)
    xx.xx_apply_vjp(PLAN, c(4), 4, w(4), 4, ct, 6, c(6), None, c(4), S)
    xx.xx_strain_derivative(PLAN, ct, wt, 6, f64(9), f64(1), S)
    xx.xx_strain_derivative(PLAN, ct, wt, 6, f64(9), None, S)
    xx.xx_energy_from_vx_noalloc(NK, 6, NPW, T(NK, dtype=torch.int32), ct, wt, vx, f64(2), S)
    plan = types.SimpleNamespace(handle=PLAN)
    xx.xx_run_many([dict(plan=plan, c_occ=ct, w_occ=w(4), c_tgt=ct, w_tgt=wt, vx_out=vx,
                         ex_out=f64(2), ld_occ=6),
                    dict(plan=plan, c_occ=c(4), w_occ=w(4), c_tgt=ct, vx_out=vx)], S)
    assert lib.calls == ["xx_apply"] * 5 + [
        "xx_energy", "xx_apply_range", "xx_energy_range", "xx_energy_from_vx",
        "xx_energy_from_vx_range", "xx_apply_backward", "xx_apply_backward", "xx_apply_vjp",
        "xx_apply_vjp", "xx_strain_derivative", "xx_strain_derivative",
        "xx_energy_from_vx_noalloc", "xx_run_many"]


@pytest.mark.parametrize("case", [
    "complex64 orbitals", "float32 occupations", "too few occupied bands", "too few k-points",
    "wrong basis length", "host tensor", "strided tensor", "short energy output",
    "short range targets", "int64 basis sizes", "short vjp output", "short strain output",
])
def test_bad_arguments_raise_before_the_library(lib, case):
    ct, vx = c(6), c(6)
    calls = {
        "complex64 orbitals": lambda: xx.xx_apply(PLAN, c(4, dtype=torch.complex64), 4, w(4), 4,
                                                  ct, 6, vx, S),
        "float32 occupations": lambda: xx.xx_apply(PLAN, c(4), 4, w(4, dtype=torch.float32), 4,
                                                   ct, 6, vx, S),
        "too few occupied bands": lambda: xx.xx_apply(PLAN, c(3), 4, w(4), 4, ct, 6, vx, S),
        "too few k-points": lambda: xx.xx_energy(PLAN, c(4), 4, w(4), 4, c(6, nk=NK - 1), w(6),
                                                 6, vx, f64(2), S),
        "wrong basis length": lambda: xx.xx_apply(PLAN, c(4), 4, w(4), 4, c(6, npw=NPW + 1), 6,
                                                  vx, S),
        "host tensor": lambda: xx.xx_apply(PLAN, c(4), 4, w(4), 4, ct, 6, c(6, cuda=False), S),
        "strided tensor": lambda: xx.xx_apply(PLAN, c(4, contiguous=False), 4, w(4), 4, ct, 6,
                                              vx, S),
        "short energy output": lambda: xx.xx_energy(PLAN, ct, 6, w(4), 4, ct, w(6), 6, vx,
                                                    f64(1), S),
        "short range targets": lambda: xx.xx_apply_range(PLAN, 0, 2, c(4), 4, w(4), 4,
                                                         c(6, nk=1), 6, c(6, nk=2), S),
        "int64 basis sizes": lambda: xx.xx_energy_from_vx_noalloc(
            NK, 6, NPW, T(NK, dtype=torch.int64), ct, w(6), vx, f64(2), S),
        "short vjp output": lambda: xx.xx_apply_vjp(PLAN, ct, 6, w(4), 4, ct, 6, c(6), c(6),
                                                    c(3), S),
        "short strain output": lambda: xx.xx_strain_derivative(PLAN, ct, w(6), 6, f64(8), None, S),
    }
    with pytest.raises(ValueError):
        calls[case]()
    assert lib.calls == []


def test_invalid_plan_is_left_to_the_library(lib):
    """A null handle skips the size checks; the library reports it."""
    xx.xx_apply(None, c(1), 1, w(1), 1, c(1), 1, c(1), S)
    assert lib.calls == ["xx_apply"]
