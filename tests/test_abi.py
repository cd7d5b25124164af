"""C-ABI checks that need no GPU: the library builds and loads, exports every
symbol include/xx.h declares, and rejects bad arguments before any GPU work."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1111_0716_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_0716_gb300 import xx
    return xx


def declared_symbols():
    with open(os.path.join(ROOT, "include", "xx.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(xx_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("xx_create", "xx_destroy", "xx_apply", "xx_energy", "xx_apply_backward",
              "xx_sync", "xx_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(xx_\w+)", out))
    for n in declared_symbols():
        assert n in exported, n
        assert hasattr(lib.load(), n)
    assert set(lib.EXPORTS) == set(declared_symbols())


def test_status_strings(lib):
    for code in range(-8, 1):
        s = lib.xx_status_string(code)
        assert isinstance(s, str) and s and s != "unknown status"
    assert lib.xx_status_string(-99) == "unknown status"


def _create(lib, wl, grid=None, kernel=None, mu=None, prec=0):
    return lib.xx_create(wl.lattice, wl.grid if grid is None else grid, wl.kfrac, wl.npw,
                         wl.miller, wl.kernel if kernel is None else kernel,
                         wl.mu if mu is None else mu, prec)


def _status(fn):
    from paper_1111_0716_gb300 import xx
    try:
        fn()
    except xx.XXError as e:
        return e.status
    return 0


def test_rejects_bad_arguments_before_gpu_work(lib):
    wl = synth.tiny_cubic()
    assert _status(lambda: _create(lib, wl, grid=(25, 25, 25))) == -2        # unsupported length
    assert _status(lambda: _create(lib, wl, grid=(24, 32, 50))) == -2        # one length unsupported
    assert _status(lambda: _create(lib, wl, grid=(24, 25, 24))) == -2        # one length unsupported
    assert _status(lambda: _create(lib, wl, kernel=7)) == -1
    assert _status(lambda: _create(lib, wl, mu=0.0)) == -1                   # screened needs mu > 0
    assert _status(lambda: _create(lib, wl, mu=float("nan"))) == -1
    assert _status(lambda: _create(lib, wl, prec=3)) == -1
    bad = wl.replace(npw=np.array([wl.npw_max + 1], dtype=np.int32))
    assert _status(lambda: _create(lib, bad)) == -1
    flat = wl.replace(lattice=np.zeros((3, 3)))
    assert _status(lambda: _create(lib, flat)) == -1


def test_rejects_grids_with_codensity_wrap_around(lib):
    # 48^3 basis (n_max = 9) on a 24^3 grid: 24 < 4*9 + 1
    wl = synth.sweep_cell(2)
    assert _status(lambda: _create(lib, wl, grid=(24, 24, 24))) == -3
    # n_max = 6 on 24: 24 < 25 is rejected, on 32: 32 >= 25 passes the check
    wl6 = synth.sweep_cell(0)
    assert int(wl6.n_max().max()) == 6
    assert _status(lambda: _create(lib, wl6, grid=(24, 24, 24))) == -3


def test_three_lengths_are_checked_on_the_callers_grid(lib):
    """Three different lengths run on a raised grid (24 x 32 x 40 -> 24 x 40 x 40), but
    wrap-around is judged on the caller's lengths: n_max = 8 along the second axis needs
    33 points, so 32 there is rejected although the raised 40 would hold it."""
    wl = synth.tiny_cubic()
    mil = wl.miller.copy()
    mil[0, 0, 1] = 8
    bad = wl.replace(miller=mil)
    assert _status(lambda: _create(lib, bad, grid=(24, 32, 40))) == -3
    assert _status(lambda: _create(lib, bad, grid=(24, 36, 40))) != -3


def test_null_plan_and_pointers(lib):
    L = lib.load()
    assert L.xx_apply(None, None, 0, None, 0, None, 0, None, None) == -1
    assert L.xx_apply_range(None, 0, 1, None, 0, None, 0, None, 0, None, None) == -1
    assert L.xx_energy(None, None, 0, None, 0, None, None, 0, None, None, None) == -1
    assert L.xx_apply_backward(None, None, None, 0, None, 1.0, None, None, None) == -1
    assert L.xx_sync(None, None, 1.0) == -1
    assert L.xx_set_batch(None, 1, 1) == -1
    assert L.xx_plan_info(None, None) == -1
    assert L.xx_destroy(None) == 0
    assert L.xx_create(None, None, None, 0, None, None, 0, None, 0, 0.0, 0, 0) == -1


def test_no_device_is_reported_without_a_gpu(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    wl = synth.tiny_cubic()
    assert _status(lambda: _create(lib, wl)) == -8
    # three different lengths pass the grid checks and reach the device query
    assert _status(lambda: _create(lib, wl, grid=(24, 32, 48))) == -8


def test_exact_grid_is_the_smallest_admissible_supported_length(lib):
    """xx_exact_grid: the smallest supported N with N >= 4 n_max + 1 on every axis."""
    supported = (24, 32, 36, 40, 48, 54, 60, 64, 72, 80, 96, 108)
    for nm in [(0, 0, 0), (4, 4, 4), (5, 4, 4), (7, 7, 7), (7, 9, 8), (14, 14, 14), (14, 12, 13),
               (15, 15, 15), (23, 1, 1), (26, 1, 1)]:
        need = 4 * max(nm) + 1
        assert lib.xx_exact_grid(nm) == min(n for n in supported if n >= need)
    # the workloads' grids are admissible, and their smallest exact grids are smaller
    for wl, n in [(synth.tiny_cubic(), 24), (synth.beta_boron(), 60)]:
        nm = wl.n_max()
        assert lib.xx_exact_grid(nm) == n
        assert wl.grid[0] >= 4 * nm.max() + 1
    assert _status(lambda: lib.xx_exact_grid((27, 0, 0))) == -2
    assert _status(lambda: lib.xx_exact_grid((-1, 0, 0))) == -1


def test_binding_has_a_function_for_every_entry_point(lib):
    """The Python binding is thin: one function per C entry point, same name."""
    for n in declared_symbols():
        assert callable(getattr(lib, n, None)), n


def test_exact_grid3_is_the_fewest_point_admissible_grid(lib):
    """xx_exact_grid3 against a brute-force search over every supported grid with two
    equal lengths (the shape the transforms run on)."""
    import itertools
    supported = (24, 32, 36, 40, 48, 54, 60, 64, 72, 80, 96, 108)
    for nm in [(0, 0, 0), (4, 4, 4), (7, 9, 8), (5, 5, 6), (14, 12, 13), (4, 9, 4), (9, 4, 4),
               (22, 3, 3), (26, 1, 26)]:
        need = [4 * v + 1 for v in nm]
        cands = [g for g in itertools.product(supported, repeat=3)
                 if all(g[i] >= need[i] for i in range(3))
                 and (g[0] == g[1] or g[0] == g[2] or g[1] == g[2])]
        best = min(g[0] * g[1] * g[2] for g in cands)
        got = lib.xx_exact_grid3(nm)
        assert got in cands and got[0] * got[1] * got[2] == best, (nm, got)
    assert _status(lambda: lib.xx_exact_grid3((27, 0, 0))) == -2
    assert _status(lambda: lib.xx_exact_grid3((0, -1, 0))) == -1
