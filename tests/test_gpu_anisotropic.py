"""FFT grids of different lengths per axis, against the FP64 oracle in both
precisions.  Two of the three equal: the plan relabels the axes so the equal pair
spans its planes -- a tetragonal cell on N x N x M with a k-mesh (the pair symmetry
across k-points), and sheared cells whose equal lengths are on axes (1, 3) and
(2, 3), so both relabellings run.  Three different lengths: the plan runs on a
grid raised to two equal lengths, and the oracle on the caller's grid -- an
orthorhombic cell with a k-mesh and a sheared Gamma cell.  The relabelling must not
change results: the same cell passed with its axes already in the plan's order
gives the same V_x c, E_x and strain derivative."""
import math

import numpy as np
import pytest

from paper_1111_0716_gb300 import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    return gu.need_gpu()


def tetragonal():
    return synth.make_workload("tetra-24x24x32", np.diag([10.0, 10.0, 13.3]), (24, 24, 32),
                               synth.monkhorst_pack(2), math.pi, 4, 6, [1.0, 1.0, 0.75, 0.3], 71)


def sheared_13():
    lat = np.array([[10.0, 0.0, 0.0], [1.5, 13.3, 0.0], [0.8, -1.1, 10.0]])
    return synth.make_workload("sheared-24x32x24", lat, (24, 32, 24), np.zeros((1, 3)), math.pi,
                               5, 6, [1.0] * 4 + [0.5], 72)


def sheared_23():
    lat = np.array([[16.0, 0.0, 0.0], [1.2, 10.0, 0.0], [-0.9, 0.7, 10.0]])
    return synth.make_workload("sheared-40x24x24", lat, (40, 24, 24), np.zeros((1, 3)), math.pi,
                               5, 5, [1.0] * 5, 73)


def orthorhombic():
    # n_max = 5, 6, 8 per axis: 24 x 32 x 40 is admissible; raised to 24 x 40 x 40
    return synth.make_workload("ortho-24x32x40", np.diag([10.0, 13.3, 16.6]), (24, 32, 40),
                               synth.monkhorst_pack(2), math.pi, 4, 6, [1.0, 1.0, 0.75, 0.3], 74)


def sheared_3lengths():
    # raised to 36 x 48 x 36 (the pair (1, 3) gives the fewest points)
    lat = np.array([[11.0, 0.0, 0.0], [1.3, 15.0, 0.0], [-0.6, 0.9, 13.0]])
    return synth.make_workload("sheared-32x48x36", lat, (32, 48, 36), np.zeros((1, 3)), math.pi,
                               5, 6, [1.0] * 4 + [0.5], 75)


# cell -> the grid the transforms run on
CELLS = {"tetra": (tetragonal, (24, 24, 32)), "sheared13": (sheared_13, (24, 32, 24)),
         "sheared23": (sheared_23, (40, 24, 24)), "ortho": (orthorhombic, (24, 40, 40)),
         "sheared3": (sheared_3lengths, (36, 48, 36))}


@pytest.mark.parametrize("name", sorted(CELLS))
@pytest.mark.parametrize("prec,tol", [(0, gu.FP32_TOL), (1, gu.FP64_TOL)])
def test_anisotropic_grid_matches_oracle(gpu, oracle_mod, name, prec, tol):
    make, runs_on = CELLS[name]
    wl = make()
    assert np.all(4 * wl.n_max() + 1 <= np.array(wl.grid))
    ref = oracle_mod.apply(wl)
    e_ref, _ = oracle_mod.energy_from_vx(wl, ref)
    for shared in (True, False):
        vx, (e, _), info = gu.run(wl, prec, shared=shared)
        w = "%s %s%s" % (name, "x".join(map(str, wl.grid)), " shared" if shared else "")
        assert gu.record(w, prec, "max|dVx|/max|Vx|", gu.rel_max(vx, ref), tol) <= tol
        assert gu.record(w, prec, "|dE_x|/|E_x|", gu.rel_err(e, e_ref), tol) <= tol
        assert tuple(info["grid"]) == runs_on


def _relabelled(wl, perm):
    """The same cell with its axes in the order perm (lattice rows, grid, Miller and
    k components)."""
    return wl.replace(lattice=np.ascontiguousarray(wl.lattice[list(perm)]),
                      grid=tuple(wl.grid[i] for i in perm),
                      kfrac=np.ascontiguousarray(wl.kfrac[:, list(perm)]),
                      miller=np.ascontiguousarray(wl.miller[:, :, list(perm)]))


@pytest.mark.parametrize("name,perm", [("sheared13", (0, 2, 1)), ("sheared23", (1, 2, 0))])
def test_relabelling_changes_nothing(gpu, name, perm):
    torch, xx = gpu
    wl = CELLS[name][0]()
    same = _relabelled(wl, perm)          # already in the plan's order: no relabelling
    assert same.grid[0] == same.grid[1]
    out = []
    for cell in (wl, same):
        vx, (e, _), _ = gu.run(cell, 1)
        plan = xx.Plan.from_workload(cell, precision=1)
        c, w = gu.dev(cell.c_tgt), gu.dev(cell.w_tgt)
        d, e2 = plan.strain_derivative(c, w)
        plan.sync(timeout_s=600.0)
        out.append((vx, e, d.cpu().numpy(), float(e2.item())))
        plan.close()
    assert gu.rel_max(out[0][0], out[1][0]) <= 1e-12
    assert abs(out[0][1] - out[1][1]) <= 1e-12 * abs(out[1][1])
    assert np.abs(out[0][2] - out[1][2]).max() <= 1e-11 * np.abs(out[1][2]).max()


def test_batched_cells_with_anisotropic_grids(gpu):
    """One launch per pass over a cubic and two anisotropic Gamma cells (pass B runs
    the z length of each batch's cell), against each cell on its own."""
    torch, xx = gpu
    cells = [synth.sweep_cell(0), sheared_13(), sheared_23()]
    plans, jobs = [], []
    for wl in cells:
        plan = xx.Plan.from_workload(wl, precision=0, workspace_cap=8 << 30)
        c = gu.dev(wl.c_tgt)
        jobs.append({"plan": plan, "c_occ": c, "ld_occ": c.shape[1], "w_occ": gu.dev(wl.w_occ),
                     "c_tgt": c, "w_tgt": gu.dev(wl.w_tgt), "vx_out": torch.empty_like(c),
                     "ex_out": torch.empty(2, dtype=torch.float64, device="cuda")})
        plans.append(plan)
    xx.xx_run_batched(jobs)
    torch.cuda.synchronize()
    for wl, job, plan in zip(cells, jobs, plans):
        single = xx.Plan.from_workload(wl, precision=0, workspace_cap=8 << 30)
        c = gu.dev(wl.c_tgt)
        ex, vx = single.energy(c, gu.dev(wl.w_occ), c, gu.dev(wl.w_tgt), shared=True)
        single.sync(timeout_s=600.0)
        assert gu.rel_max(job["vx_out"].cpu().numpy(), vx.cpu().numpy()) <= 1e-12
        single.close()
        plan.close()
