"""The six uneven sweep cells (grids 32^3 ... 80^3, 16 ... 96 bands, Gamma) in one
launch per band-pair pass (xx_run_batched), against each cell run on its own
(xx_energy) and against the FP64 oracle on sampled targets, in both precisions
and with both kernels; several rounds when a plan's workspace cap is small."""
import numpy as np
import pytest

from paper_1111_0716_gb300 import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    return gu.need_gpu()


def single(xx, torch, wl, prec, cap):
    """The cell on its own (xx_energy) with the same workspace cap, hence the same batches."""
    plan = xx.Plan.from_workload(wl, precision=prec, workspace_cap=cap)
    c = gu.dev(wl.c_tgt)
    ex, vx = plan.energy(c, gu.dev(wl.w_occ), c, gu.dev(wl.w_tgt), shared=True)
    plan.sync(timeout_s=600.0)
    out = vx.cpu().numpy(), float(ex[0].item())
    plan.close()
    return out


def jobs_for(xx, torch, cells, prec, caps=None):
    plans, jobs = [], []
    for i, wl in enumerate(cells):
        cap = caps[i] if caps else 48 << 30
        plan = xx.Plan.from_workload(wl, precision=prec, workspace_cap=cap)
        c = gu.dev(wl.c_tgt)
        jobs.append({"plan": plan, "c_occ": c, "ld_occ": c.shape[1], "w_occ": gu.dev(wl.w_occ),
                     "c_tgt": c, "w_tgt": gu.dev(wl.w_tgt), "vx_out": torch.empty_like(c),
                     "ex_out": torch.empty(2, dtype=torch.float64, device="cuda")})
        plans.append(plan)
    return plans, jobs


@pytest.mark.parametrize("kernel", [synth.KERNEL_HSE, synth.KERNEL_COULOMB])
@pytest.mark.parametrize("prec", [0, 1])
def test_batched_sweep_matches_single_cells_and_oracle(gpu, oracle_mod, prec, kernel):
    torch, xx = gpu
    cells = [synth.sweep_cell(i, kernel) for i in range(len(synth.SWEEP_GRIDS))]
    plans, jobs = jobs_for(xx, torch, cells, prec)
    xx.xx_run_batched(jobs)
    torch.cuda.synchronize()
    tol = gu.FP32_TOL if prec == 0 else gu.FP64_TOL
    for wl, job, plan in zip(cells, jobs, plans):
        plan.sync(timeout_s=600.0)
        vx = job["vx_out"].cpu().numpy()
        e = float(job["ex_out"][0].item())
        # the same batches as the single-cell path: the same sums in the same order
        ref_vx, ref_e = single(xx, torch, wl, prec, 48 << 30)
        assert gu.rel_max(vx, ref_vx) <= 1e-12
        assert abs(e - ref_e) <= 1e-12 * abs(ref_e)
        sel = [(0, 0), (0, wl.n_tgt - 1)]
        ref = oracle_mod.apply(wl, sel=sel)
        got = np.stack([vx[k, a] for k, a in sel])
        w = "batched " + wl.name
        assert gu.record(w, prec, "max|dVx|/max|Vx| (2 targets)", gu.rel_max(got, ref), tol) <= tol
        plan.close()


def test_batched_rounds_and_requirements(gpu):
    """A small workspace cap on two plans splits their batches over several rounds
    (one launch per pass and round); the result does not change.  Plans with
    several k-points, mixed precisions or a plan given twice are refused."""
    torch, xx = gpu
    cells = [synth.sweep_cell(i) for i in (0, 3, 5)]
    plans, jobs = jobs_for(xx, torch, cells, 0)
    xx.xx_run_batched(jobs)
    torch.cuda.synchronize()
    one = [j["vx_out"].cpu().numpy() for j in jobs]
    for p in plans:
        p.close()
    caps = [48 << 30, 1 << 30, 2 << 30]
    plans, jobs = jobs_for(xx, torch, cells, 0, caps)
    xx.xx_run_batched(jobs)
    torch.cuda.synchronize()
    for wl, cap, a, j in zip(cells, caps, one, jobs):
        got = j["vx_out"].cpu().numpy()
        ref, _ = single(xx, torch, wl, 0, cap)
        assert gu.rel_max(got, ref) <= 1e-12          # same batches as the single cell
        assert gu.rel_max(got, a) <= 1e-6             # other batches: FP32 sums regrouped
    with pytest.raises(xx.XXError):
        xx.xx_run_batched([jobs[0], dict(jobs[0])])
    for p in plans:
        p.close()
    wl = synth.make_workload("k2", synth.cubic_lattice(10.0), (24,) * 3, synth.monkhorst_pack(2),
                             2.0, 2, 2, [1.0, 1.0], 5)
    plans, jobs = jobs_for(xx, torch, [wl], 0)
    with pytest.raises(xx.XXError):
        xx.xx_run_batched(jobs)
    for p in plans:
        p.close()
    p32, j32 = jobs_for(xx, torch, [cells[0]], 0)
    p64, j64 = jobs_for(xx, torch, [cells[1]], 1)
    with pytest.raises(xx.XXError):
        xx.xx_run_batched(j32 + j64)
    for p in p32 + p64:
        p.close()
