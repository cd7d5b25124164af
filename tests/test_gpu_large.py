"""Full-size workloads in the launch configuration the benchmark times.

The CUDA path runs the whole operator; the oracle computes sampled targets one
by one (each target needs every occupied band of every q); properties that
hold at any size (Hermiticity of <c_b|V_x c_a> at every k) cover the rest; an
FP64 GPU slice checks the all-FP64 path at the same size.
"""
import numpy as np
import pytest

from paper_1111_0716_gb300 import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    return gu.need_gpu()


def fp64_target_slice(xx, wl, k, a):
    plan = xx.Plan.from_workload(wl, precision=1)
    co, wo = gu.dev(wl.c_occ), gu.dev(wl.w_occ)
    ct = gu.dev(wl.c_tgt[k:k + 1, a:a + 1])
    vx = plan.apply_range(k, 1, co, wo, ct)
    plan.sync(timeout_s=600.0)
    out = vx.cpu().numpy()[0, 0]
    plan.close()
    return out


def fp32_target_slice(xx, wl, k, a, tj):
    """V_x c of target (k, a) alone, FP32-mixed, occupied batches tj bands wide."""
    plan = xx.Plan.from_workload(wl, precision=0)
    plan.set_batch(1, tj)
    co, wo = gu.dev(wl.c_occ), gu.dev(wl.w_occ)
    vx = plan.apply_range(k, 1, co, wo, gu.dev(wl.c_tgt[k:k + 1, a:a + 1]))
    plan.sync(timeout_s=600.0)
    out = vx.cpu().numpy()[0, 0]
    plan.close()
    return out


def test_alpha_boron_48_mp444(gpu, oracle_mod):
    torch, xx = gpu
    wl = synth.alpha_boron()
    vx, (e, e_im), info = gu.run(wl, 0)
    assert abs(e_im) <= gu.FP32_TOL * abs(e)
    w = "alpha-boron 48^3 MP4x4x4 (18/24)"
    t32 = gu.FP32_TOL
    assert gu.record(w, 0, "Hermiticity defect", gu.hermitian_defect(wl.c_tgt, vx), t32) <= t32
    # sampled targets: the first band at the first k-point, an occupied band at an
    # inner k-point (it receives the role-swapped contributions of the blocks
    # q < k of multi-q batches), and the last target past the occupied set
    sel = [(0, 0), (wl.nk // 2, 0), (wl.nk - 1, wl.n_tgt - 1)]
    ref = oracle_mod.apply(wl, sel=sel)
    for (k, a), r in zip(sel, ref):
        assert gu.record(w, 0, "max|dVx|/max|Vx| target (%d,%d)" % (k, a),
                         gu.rel_max(vx[k, a], r), t32) <= t32
        d_gpu = np.vdot(wl.c_tgt[k, a], vx[k, a]).real
        d_ref = np.vdot(wl.c_tgt[k, a], r).real
        assert gu.record(w, 0, "<c|Vx c> rel, target (%d,%d)" % (k, a),
                         gu.rel_err(d_gpu, d_ref), t32) <= t32
    v64 = fp64_target_slice(xx, wl, *sel[1])
    assert gu.record(w, 1, "max|dVx|/max|Vx| target (%d,%d)" % sel[1], gu.rel_max(v64, ref[1]),
                     gu.FP64_TOL) <= gu.FP64_TOL
    # the smallest exact grid (32^3 for n_max = 7) gives the same operator as 48^3,
    # in both precisions
    n = xx.xx_exact_grid(wl.n_max())
    assert n == 32
    small = wl.replace(grid=(n,) * 3)
    vx32, (e32, _), _ = gu.run(small, 0)
    assert gu.rel_max(np.stack([vx32[k, a] for k, a in sel]), ref) <= gu.FP32_TOL
    assert abs(e32 - e) <= gu.FP32_TOL * abs(e)
    w64 = fp64_target_slice(xx, small, *sel[1])
    assert gu.rel_max(w64, ref[1]) <= gu.FP64_TOL


@pytest.mark.slow
def test_beta_boron_96_gamma222(gpu, oracle_mod):
    torch, xx = gpu
    wl = synth.beta_boron()
    vx, (e, e_im), info = gu.run(wl, 0)
    assert abs(e_im) <= gu.FP32_TOL * abs(e)
    w = "beta-boron 96^3 G2x2x2 (160/192)"
    t32 = gu.FP32_TOL
    assert gu.record(w, 0, "Hermiticity defect", gu.hermitian_defect(wl.c_tgt, vx), t32) <= t32
    # sampled targets: the first band at Gamma (a k = q diagonal tile), a target past
    # the occupied set at an inner k-point (every occupied band of every q, no pair
    # symmetry), and a fractionally occupied band at the zone-boundary k-point
    sel = [(0, 0), (3, wl.n_tgt - 1), (wl.nk - 1, 155)]
    refs = oracle_mod.apply(wl, sel=sel)
    for (kk, aa), r in zip(sel, refs):
        assert gu.record(w, 0, "max|dVx|/max|Vx| target (%d,%d)" % (kk, aa),
                         gu.rel_max(vx[kk, aa], r), t32) <= t32, (kk, aa)
        d_gpu = np.vdot(wl.c_tgt[kk, aa], vx[kk, aa]).real
        d_ref = np.vdot(wl.c_tgt[kk, aa], r).real
        assert gu.record(w, 0, "<c|Vx c> rel, target (%d,%d)" % (kk, aa),
                         gu.rel_err(d_gpu, d_ref), t32) <= t32
    k, a = sel[-1]
    ref = refs[-1]
    v64 = fp64_target_slice(xx, wl, k, a)
    assert gu.record(w, 1, "max|dVx|/max|Vx| target (%d,%d)" % (k, a), gu.rel_max(v64, ref),
                     gu.FP64_TOL) <= gu.FP64_TOL
    # the FP32 partial sums over an occupied batch before each FP64 add: the
    # production width (80 occupied per batch) against 8 per batch, same targets
    for (kk, aa), r in zip(sel, refs):
        for tj in (80, 8):
            v = fp32_target_slice(xx, wl, kk, aa, tj)
            assert gu.record(w, 0, "max|dVx|/max|Vx| (%d,%d), %d occ/batch" % (kk, aa, tj),
                             gu.rel_max(v, r), t32) <= t32
    # the smallest exact grid (60^3 for n_max = 14) gives the same operator as 96^3
    n = xx.xx_exact_grid(wl.n_max())
    assert n == 60
    vx60, (e60, _), _ = gu.run(wl.replace(grid=(n,) * 3), 0)
    assert gu.rel_max(vx60[k, a], ref) <= gu.FP32_TOL
    assert abs(e60 - e) <= gu.FP32_TOL * abs(e)
    assert gu.rel_max(vx60, vx) <= gu.FP32_TOL
