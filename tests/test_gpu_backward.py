"""Gradients of E_x on the GPU: dE/dc* and dE/dmu against the oracle, central
finite differences of the GPU's own FP64 energy, and the autograd Function."""
import numpy as np
import pytest

from paper_1111_0716_gb300 import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    return gu.need_gpu()


def gpu_energy(xx, torch, wl, c, mu=None, prec=1):
    plan = xx.Plan.from_workload(wl, precision=prec, mu=mu)
    ct = gu.dev(c)
    w = gu.dev(wl.w_tgt)
    ex, _ = plan.energy(ct, w, ct, w, shared=True)
    e = float(ex[0].item())
    plan.close()
    return e


@pytest.mark.parametrize("prec,tol", [(0, gu.FP32_TOL), (1, gu.FP64_TOL)])
def test_backward_matches_oracle_on_differentiation_cell(gpu, oracle_mod, prec, tol):
    torch, xx = gpu
    wl = synth.differentiation_cell()
    vx_ref = oracle_mod.apply(wl)
    dmu_ref = oracle_mod.pair_sum(wl, which=1)
    plan = xx.Plan.from_workload(wl, precision=prec)
    c, w = gu.dev(wl.c_tgt), gu.dev(wl.w_tgt)
    grad = 0.7
    dc, dmu = plan.backward(c, w, grad_ex=grad)          # recomputes V_x c
    plan.sync(timeout_s=600.0)
    peak = plan.info()["peak_workspace_bytes"]
    plan.close()
    ref = grad * 2.0 * wl.w_tgt[:, :, None] / wl.nk * vx_ref
    w = "differentiation cell 48^3 (32/32)"
    assert gu.record(w, prec, "dE/dc*: max|d|/max|ref| (f_a Vx c)", gu.rel_max(dc.cpu().numpy(), ref),
                     tol) <= tol
    assert gu.record(w, prec, "dE/dmu rel (closed form)", gu.rel_err(float(dmu.item()), grad * dmu_ref),
                     tol) <= tol
    # the backward keeps no per-pair grid: its workspace is the orbital grids, one
    # band-pair batch and the accumulators, far below n_b^2 full grids
    n3 = 48 ** 3
    bound = wl.n_tgt ** 2 * n3 * 8
    # listed with the achieved errors: the peak workspace in MB, against n_b^2 grids
    assert gu.record(w, prec, "backward peak workspace, MB (vs n_b^2 grids)", peak / 1e6,
                     bound / 1e6) < bound / 1e6


def test_dc_matches_finite_differences_of_gpu_energy(gpu):
    torch, xx = gpu
    wl = synth.tiny_cubic()
    plan = xx.Plan.from_workload(wl, precision=1)
    c, w = gu.dev(wl.c_tgt), gu.dev(wl.w_tgt)
    dc, _ = plan.backward(c, w, grad_ex=1.0, want_dmu=False)
    grad = dc.cpu().numpy()
    plan.close()
    rng = np.random.default_rng(4)
    h = 1e-4
    worst = 0.0
    for _ in range(16):
        d = rng.standard_normal(wl.c_tgt.shape) + 1j * rng.standard_normal(wl.c_tgt.shape)
        d[:, :, wl.npw[0]:] = 0
        d /= np.linalg.norm(d)
        fd = (gpu_energy(xx, torch, wl, wl.c_tgt + h * d) -
              gpu_energy(xx, torch, wl, wl.c_tgt - h * d)) / (2 * h)
        an = 2.0 * np.real(np.vdot(d, grad))
        worst = max(worst, abs(fd - an) / max(abs(an), 1e-3 * np.abs(grad).max()))
    assert gu.record("tiny cubic 24^3 (8/8, Gamma)", 1, "dE/dc* vs central FD, worst of 16", worst,
                     1e-7) <= 1e-7


def test_dmu_matches_finite_differences_of_gpu_energy(gpu):
    torch, xx = gpu
    wl = synth.tiny_cubic()
    plan = xx.Plan.from_workload(wl, precision=1)
    c, w = gu.dev(wl.c_tgt), gu.dev(wl.w_tgt)
    _, dmu = plan.backward(c, w, grad_ex=1.0, want_dc=False)
    dmu = float(dmu.item())
    plan.close()
    h = 1e-4

    def cd(step):
        return (gpu_energy(xx, torch, wl, wl.c_tgt, mu=wl.mu + step) -
                gpu_energy(xx, torch, wl, wl.c_tgt, mu=wl.mu - step)) / (2 * step)
    fd = (4 * cd(h) - cd(2 * h)) / 3
    assert gu.record("tiny cubic 24^3 (8/8, Gamma)", 1, "dE/dmu vs Richardson FD (h=1e-4)",
                     gu.rel_err(dmu, fd), 1e-8) <= 1e-8


@pytest.mark.parametrize("prec", [0, 1])
def test_autograd_function(gpu, oracle_mod, prec):
    torch, xx = gpu
    wl = synth.tiny_cubic()
    plan = xx.Plan.from_workload(wl, precision=prec)
    c = gu.dev(wl.c_tgt).requires_grad_(True)
    w = gu.dev(wl.w_tgt)
    mu = torch.tensor(wl.mu, dtype=torch.float64, requires_grad=True)
    e = xx.exchange_energy(c, w, mu, plan)
    (3.0 * e).backward()
    vx_ref = oracle_mod.apply(wl)
    e_ref, _ = oracle_mod.energy_from_vx(wl, vx_ref)
    tol = gu.FP32_TOL if prec == 0 else gu.FP64_TOL
    assert abs(float(e.item()) - e_ref) <= tol * abs(e_ref)
    # torch convention: .grad = 2 dL/dc* = 2 * 3 * (s w / N_k) V_x c
    ref = 2.0 * 3.0 * 2.0 * wl.w_tgt[:, :, None] / wl.nk * vx_ref
    assert gu.rel_max(c.grad.cpu().numpy(), ref) <= tol
    dmu_ref = oracle_mod.pair_sum(wl, which=1)
    assert abs(float(mu.grad.item()) - 3.0 * dmu_ref) <= tol * abs(3.0 * dmu_ref)
    plan.close()


def test_sync_time_limit_reports_timeout_without_cancelling(gpu):
    """A host wait with a tiny limit returns XX_ERR_TIMEOUT; a later wait completes."""
    torch, xx = gpu
    wl = synth.alpha_boron()
    plan = xx.Plan.from_workload(wl, precision=0)
    c, w = gu.dev(wl.c_tgt), gu.dev(wl.w_tgt)
    wo = gu.dev(wl.w_occ)
    vx = torch.empty_like(c)
    xx.xx_apply(plan.handle, c, c.shape[1], wo, wl.n_occ, c, c.shape[1], vx)
    with pytest.raises(xx.XXError) as ei:
        plan.sync(timeout_s=1e-4)
    assert ei.value.status == -7
    plan.sync(timeout_s=600.0)
    assert torch.isfinite(vx.abs()).all()
    plan.close()


def rhombo_mesh():
    """Rhombohedral cell with a 2x2x2 MP mesh (8 k-points, 4 bands)."""
    return synth.make_workload("rhombo24", synth.rhombohedral_lattice(7.5, 65.0), (24,) * 3,
                               synth.monkhorst_pack(2), 2.4, 4, 4, [1.0, 1.0, 0.75, 0.3], 21)


@pytest.mark.parametrize("make", [lambda: synth.sweep_cell(0), rhombo_mesh])
@pytest.mark.parametrize("prec,tol", [(0, gu.FP32_TOL), (1, 1e-12)])
def test_dmu_pair_symmetry_matches_direct_pairs(gpu, prec, tol, make):
    """dE/dmu with the pair symmetry (k = q tiles, blocks q > k counted twice) and
    with every pair transformed."""
    torch, xx = gpu
    wl = make()
    out = []
    for on in (True, False):
        plan = xx.Plan.from_workload(wl, precision=prec)
        plan.set_batch(5, 5)
        plan.set_pair_symmetry(on)
        _, dmu = plan.backward(gu.dev(wl.c_tgt), gu.dev(wl.w_tgt), grad_ex=1.0, want_dc=False)
        out.append(float(dmu.item()))
        plan.close()
    assert abs(out[0] - out[1]) <= tol * abs(out[1])


def test_device_copy_wait_expiry_is_reported(gpu):
    """A tensor copy whose bounded wait runs out (the test option announces it 16 bytes
    longer than it is) makes the CTA set the device flag and return: xx_sync reports
    XX_ERR_DEVICE_FLAG, and the same context then computes a correct result."""
    torch, xx = gpu
    wl = synth.tiny_cubic()
    c = gu.dev(wl.c_tgt)
    wo, wt = gu.dev(wl.w_occ), gu.dev(wl.w_tgt)
    plan = xx.Plan.from_workload(wl, precision=0)
    plan.set_tma_pass_b(2)
    xx.xx_set_option(plan.handle, xx.XX_OPT_TEST_WAIT_EXPIRY, 1)
    plan.energy(c, wo, c, wt, shared=True)
    with pytest.raises(xx.XXError) as ei:
        plan.sync(timeout_s=120.0)
    assert ei.value.status == -6            # XX_ERR_DEVICE_FLAG, cleared by the report
    xx.xx_set_option(plan.handle, xx.XX_OPT_TEST_WAIT_EXPIRY, 0)
    ex, vx = plan.energy(c, wo, c, wt, shared=True)
    plan.sync(timeout_s=120.0)
    ref, (e_ref, _), _ = gu.run(wl, 0)
    assert gu.rel_max(vx.cpu().numpy(), ref) <= 1e-6
    assert abs(float(ex[0].item()) - e_ref) <= 1e-6 * abs(e_ref)
    plan.close()
