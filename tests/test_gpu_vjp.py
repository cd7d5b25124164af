"""Vector-Jacobian product of V_x c (xx_apply_vjp) against finite differences of
the FP64 oracle's forward application, and the autograd Function built on it.

With L = Re <p|V_x[c_occ] c_tgt>, L is linear in c_tgt and quadratic
(sesquilinear) in c_occ, so central differences are exact up to rounding."""
import numpy as np
import pytest

from paper_1111_0716_gb300 import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    return gu.need_gpu()


def rhombo24(seed=21):
    return synth.make_workload("rhombo24", synth.rhombohedral_lattice(7.5, 65.0), (24,) * 3,
                               synth.monkhorst_pack(2), 2.4, 4, 6, [1.0, 1.0, 0.75, 0.3], seed)


def masked_random(rng, wl, shape):
    d = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    for k in range(wl.nk):
        d[k, :, wl.npw[k]:] = 0
    return d / np.linalg.norm(d)


def gpu_vjp(xx, wl, ybar, prec):
    plan = xx.Plan.from_workload(wl, precision=prec)
    gt, go = plan.vjp(gu.dev(wl.c_occ), gu.dev(wl.w_occ), gu.dev(wl.c_tgt), gu.dev(ybar))
    plan.sync(timeout_s=600.0)
    out = gt.cpu().numpy(), go.cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("make", [rhombo24, synth.tiny_cubic])
def test_vjp_matches_finite_differences_of_oracle(gpu, oracle_mod, make):
    torch, xx = gpu
    wl = make()
    rng = np.random.default_rng(3)
    pvec = masked_random(rng, wl, wl.c_tgt.shape)
    gt, go = gpu_vjp(xx, wl, 0.5 * pvec, 1)             # dL/dy* = p / 2

    def loss(c_occ=None, c_tgt=None):
        vx = oracle_mod.apply(wl, c_occ=c_occ, c_tgt=c_tgt)
        return float(np.real(np.vdot(pvec, vx)))
    h = 1e-3
    worst_t = worst_o = 0.0
    for _ in range(4):
        d = masked_random(rng, wl, wl.c_tgt.shape)
        fd = (loss(c_tgt=wl.c_tgt + h * d) - loss(c_tgt=wl.c_tgt - h * d)) / (2 * h)
        an = 2.0 * np.real(np.vdot(d, gt))
        worst_t = max(worst_t, abs(fd - an) / max(abs(an), np.abs(gt).max()))
        d = masked_random(rng, wl, wl.c_occ.shape)
        fd = (loss(c_occ=wl.c_occ + h * d) - loss(c_occ=wl.c_occ - h * d)) / (2 * h)
        an = 2.0 * np.real(np.vdot(d, go))
        worst_o = max(worst_o, abs(fd - an) / max(abs(an), np.abs(go).max()))
    w = "VJP " + wl.name
    assert gu.record(w, 1, "dL/dc_tgt* vs oracle FD, worst of 4", worst_t, 1e-9) <= 1e-9
    assert gu.record(w, 1, "dL/dc_occ* vs oracle FD, worst of 4", worst_o, 1e-9) <= 1e-9


def test_vjp_mixed_precision_matches_fp64(gpu):
    torch, xx = gpu
    wl = rhombo24()
    ybar = masked_random(np.random.default_rng(5), wl, wl.c_tgt.shape)
    gt64, go64 = gpu_vjp(xx, wl, ybar, 1)
    gt32, go32 = gpu_vjp(xx, wl, ybar, 0)
    assert gu.record("VJP " + wl.name, 0, "dL/dc_tgt* vs FP64 path", gu.rel_max(gt32, gt64),
                     gu.FP32_TOL) <= gu.FP32_TOL
    assert gu.record("VJP " + wl.name, 0, "dL/dc_occ* vs FP64 path", gu.rel_max(go32, go64),
                     gu.FP32_TOL) <= gu.FP32_TOL


def test_autograd_apply_function(gpu, oracle_mod):
    torch, xx = gpu
    wl = rhombo24()
    plan = xx.Plan.from_workload(wl, precision=1)
    rng = np.random.default_rng(11)
    pvec = masked_random(rng, wl, wl.c_tgt.shape)
    c_occ = gu.dev(wl.c_occ).requires_grad_(True)
    c_tgt = gu.dev(wl.c_tgt).requires_grad_(True)
    y = xx.exchange_apply(c_occ, gu.dev(wl.w_occ), c_tgt, plan)
    ref = oracle_mod.apply(wl)
    assert gu.rel_max(y.detach().cpu().numpy(), ref) <= gu.FP64_TOL
    loss = torch.real(torch.sum(torch.conj(gu.dev(pvec)) * y))
    loss.backward()
    gt, go = gpu_vjp(xx, wl, 0.5 * pvec, 1)
    # torch convention: .grad = 2 dL/dz*
    assert gu.rel_max(c_tgt.grad.cpu().numpy(), 2 * gt) <= 1e-12
    assert gu.rel_max(c_occ.grad.cpu().numpy(), 2 * go) <= 1e-12
    plan.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-6), (1, 1e-12)])
def test_fused_vjp_matches_separate_parts(gpu, prec, tol):
    """Both gradients from two transforms per pair (default) against the target and
    occupied parts computed by separate calls (three transforms per pair)."""
    torch, xx = gpu
    wl = rhombo24()
    rng = np.random.default_rng(7)
    ybar = masked_random(rng, wl, wl.c_tgt.shape)
    fused = gpu_vjp(xx, wl, ybar, prec)
    plan = xx.Plan.from_workload(wl, precision=prec)
    xx.xx_set_option(plan.handle, xx.XX_OPT_FUSED_VJP, 0)
    co, wo, ct, yb = gu.dev(wl.c_occ), gu.dev(wl.w_occ), gu.dev(wl.c_tgt), gu.dev(ybar)
    gt, _ = plan.vjp(co, wo, ct, yb, want_occ=False)
    _, go = plan.vjp(co, wo, ct, yb, want_tgt=False)
    plan.sync(timeout_s=600.0)
    sep = gt.cpu().numpy(), go.cpu().numpy()
    plan.close()
    assert gu.rel_max(fused[0], sep[0]) <= tol
    assert gu.rel_max(fused[1], sep[1]) <= tol


def test_fused_vjp_falls_back_without_room(gpu):
    """XX_OPT_ACC_LIMIT_MB = 0 leaves no room for the occupied accumulators of every
    k-point: xx_apply_vjp computes the two parts one after the other, same result."""
    torch, xx = gpu
    wl = rhombo24()
    rng = np.random.default_rng(11)
    ybar = masked_random(rng, wl, wl.c_tgt.shape)
    fused = gpu_vjp(xx, wl, ybar, 1)
    plan = xx.Plan.from_workload(wl, precision=1)
    xx.xx_set_option(plan.handle, xx.XX_OPT_ACC_LIMIT_MB, 0)
    gt, go = plan.vjp(gu.dev(wl.c_occ), gu.dev(wl.w_occ), gu.dev(wl.c_tgt), gu.dev(ybar))
    plan.sync(timeout_s=600.0)
    assert gu.rel_max(gt.cpu().numpy(), fused[0]) <= 1e-12
    assert gu.rel_max(go.cpu().numpy(), fused[1]) <= 1e-12
    plan.close()


def test_vjp_with_shared_grids_matches_separate_arrays(gpu):
    """Occupied bands passed as the leading target bands (ld_occ = n_tgt, the grids
    then stored occupied-first) against a separate occupied array, FP64."""
    torch, xx = gpu
    wl = rhombo24()
    rng = np.random.default_rng(5)
    ybar = gu.dev(masked_random(rng, wl, wl.c_tgt.shape))
    ref = gpu_vjp(xx, wl, ybar.cpu().numpy(), 1)
    plan = xx.Plan.from_workload(wl, precision=1)
    ct, wo = gu.dev(wl.c_tgt), gu.dev(wl.w_occ)
    gt = torch.empty_like(ct)
    go = torch.empty((wl.nk, wl.n_occ, wl.npw_max), dtype=ct.dtype, device=ct.device)
    xx.xx_apply_vjp(plan.handle, ct, wl.n_tgt, wo, wl.n_occ, ct, wl.n_tgt, ybar, gt, go)
    plan.sync(timeout_s=600.0)
    assert gu.rel_max(gt.cpu().numpy(), ref[0]) <= 1e-12
    assert gu.rel_max(go.cpu().numpy(), ref[1]) <= 1e-12
    plan.close()
