"""Real-orbital Gamma path (plan option XX_OPT_REAL_GAMMA) through the C ABI.

With orbitals that are real in real space (c(-G) = conj c(G)) at k = q = Gamma,
two occupied bands share one transform.  The result is the same operator, so it
is compared with the FP64 oracle (mixed precision 1e-5, FP64 1e-11) and with the
general path of the same library (same precision, agreement to rounding).
"""
import numpy as np
import pytest

from paper_1111_0716_gb300 import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    return gu.need_gpu()


@pytest.fixture(scope="module")
def oracle_refs(oracle_mod):
    cache = {}

    def get(name, wl):
        if name not in cache:
            cache[name] = oracle_mod.apply(wl)
        return cache[name]
    return get


def run(xx, wl, prec, real, sym=True, batch=None, shared=True):
    """(vx numpy, E_x) of the CUDA path with the given options."""
    plan = xx.Plan.from_workload(wl, precision=prec)
    if batch:
        plan.set_batch(*batch)
    plan.set_pair_symmetry(sym)
    plan.set_real_gamma(real)
    ct = gu.dev(wl.c_tgt)
    wo = gu.dev(wl.w_occ)
    wt = gu.dev(wl.w_tgt)
    if shared:
        ex, vx = plan.energy(ct, wo, ct, wt, shared=True)
    else:
        ex, vx = plan.energy(gu.dev(wl.c_occ), wo, ct, wt)
    plan.sync(timeout_s=600.0)
    out = vx.cpu().numpy(), float(ex[0].item())
    plan.close()
    return out


CELLS = {
    "cubic24_7o9t": synth.real_tiny_cubic,
    "cubic24_coulomb": lambda: synth.real_tiny_cubic(kernel=synth.KERNEL_COULOMB),
    "alpha48_18o24t": synth.real_alpha_cell,
}


@pytest.mark.parametrize("name", sorted(CELLS))
@pytest.mark.parametrize("sym", [True, False])
@pytest.mark.parametrize("prec,tol", [(0, gu.FP32_TOL), (1, gu.FP64_TOL)])
def test_real_gamma_matches_oracle(gpu, oracle_mod, oracle_refs, name, sym, prec, tol):
    torch, xx = gpu
    wl = CELLS[name]()
    ref = oracle_refs(name, wl)
    e_ref, _ = oracle_mod.energy_from_vx(wl, ref)
    vx, e = run(xx, wl, prec, True, sym=sym, batch=(3, 2))
    w = "real Gamma %s%s" % (name, " sym" if sym else "")
    assert gu.record(w, prec, "max|dVx|/max|Vx|", gu.rel_max(vx, ref), tol) <= tol
    assert gu.record(w, prec, "|dE_x|/|E_x|", gu.rel_err(e, e_ref), tol) <= tol


@pytest.mark.parametrize("prec,tol", [(0, gu.FP32_TOL), (1, gu.FP64_TOL)])
def test_real_gamma_separate_occupied_array(gpu, oracle_mod, oracle_refs, prec, tol):
    """Occupied orbitals passed as their own array (no grid sharing, no pair symmetry)."""
    torch, xx = gpu
    wl = synth.real_tiny_cubic()
    ref = oracle_refs("cubic24_7o9t", wl)
    vx, _ = run(xx, wl, prec, True, shared=False)
    assert gu.rel_max(vx, ref) <= tol


@pytest.mark.parametrize("batch", [(1, 1), (2, 1), (1, 3), (5, 3), (9, 4), (0, 0)])
def test_real_gamma_batch_shapes_agree(gpu, batch):
    """Tile shapes (odd, one band, larger than the band count) change only rounding order."""
    torch, xx = gpu
    wl = synth.real_tiny_cubic(n_occ=7, n_tgt=9)
    ref, e_ref = run(xx, wl, 1, False, sym=False)
    vx, e = run(xx, wl, 1, True, batch=batch)
    assert gu.rel_max(vx, ref) <= 1e-12
    assert abs(e - e_ref) <= 1e-12 * abs(e_ref)


@pytest.mark.parametrize("n_occ", [1, 2, 3])
def test_real_gamma_few_occupied(gpu, oracle_mod, n_occ):
    """One slot with a single band, one full slot, and a full plus a half slot."""
    torch, xx = gpu
    wl = synth.real_tiny_cubic(n_occ=n_occ, n_tgt=4)
    ref = oracle_mod.apply(wl)
    for sym in (True, False):
        vx, _ = run(xx, wl, 1, True, sym=sym)
        assert gu.rel_max(vx, ref) <= gu.FP64_TOL


@pytest.mark.parametrize("prec,tol", [(0, 2e-5), (1, 1e-11)])
def test_real_gamma_backward_and_strain(gpu, prec, tol):
    """dE/dc*, dE/dmu and dE/deps of the real path against the general path."""
    torch, xx = gpu
    wl = synth.real_tiny_cubic(n_occ=7, n_tgt=7)
    c = gu.dev(wl.c_tgt)
    w = gu.dev(wl.w_tgt)
    out = {}
    for real in (True, False):
        plan = xx.Plan.from_workload(wl, precision=prec)
        plan.set_batch(3, 2)
        plan.set_real_gamma(real)
        dc, dmu = plan.backward(c, w, grad_ex=1.0)
        d, e = plan.strain_derivative(c, w)
        plan.sync(timeout_s=600.0)
        out[real] = (dc.cpu().numpy(), float(dmu.item()), d.cpu().numpy(), float(e.item()))
        plan.close()
    a, b = out[True], out[False]
    assert gu.rel_max(a[0], b[0]) <= tol
    assert abs(a[1] - b[1]) <= tol * abs(b[1])
    assert np.abs(a[2] - b[2]).max() <= tol * np.abs(b[2]).max()
    assert abs(a[3] - b[3]) <= tol * abs(b[3])


def test_real_gamma_vjp_takes_general_path(gpu):
    """The VJP's cotangent is complex: the option must not change it."""
    torch, xx = gpu
    wl = synth.real_tiny_cubic(n_occ=5, n_tgt=6)
    rng = np.random.Generator(np.random.PCG64(7))
    ybar = rng.standard_normal(wl.c_tgt.shape) + 1j * rng.standard_normal(wl.c_tgt.shape)
    for k in range(wl.nk):
        ybar[k, :, wl.npw[k]:] = 0.0
    outs = []
    for real in (True, False):
        plan = xx.Plan.from_workload(wl, precision=1)
        plan.set_real_gamma(real)
        gt, go = plan.vjp(gu.dev(wl.c_occ), gu.dev(wl.w_occ), gu.dev(wl.c_tgt), gu.dev(ybar))
        plan.sync(timeout_s=600.0)
        outs.append((gt.cpu().numpy(), go.cpu().numpy()))
        plan.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_real_gamma_option_needs_a_closed_gamma_basis(gpu):
    torch, xx = gpu
    plan = xx.Plan.from_workload(synth.alpha_boron(), precision=0)   # 4x4x4 mesh
    with pytest.raises(xx.XXError):
        plan.set_real_gamma(True)
    plan.set_real_gamma(False)
    plan.close()
    wl = synth.real_tiny_cubic()
    n = int(wl.npw[0])
    keep = [g for g in range(n) if tuple(wl.miller[0, g]) != (1, 0, 0)]   # drop one G, keep -G
    miller = wl.miller[:, keep]
    half = xx.Plan(wl.lattice, wl.grid, wl.kfrac, np.array([len(keep)], dtype=np.int32), miller,
                   kernel=wl.kernel, mu=wl.mu, precision=0)
    with pytest.raises(xx.XXError):
        half.set_real_gamma(True)
    half.close()
    ok = xx.Plan.from_workload(wl, precision=0)
    ok.set_real_gamma(True)
    ok.close()


@pytest.mark.parametrize("make", [synth.real_tiny_cubic, synth.real_alpha_cell])
def test_real_gamma_staged_passes_match(gpu, make):
    """The real-orbital path with pass A fed by bulk copies and the tensor-copy pass B
    (forced on) against the unstaged kernels, FP32, odd tiles."""
    torch, xx = gpu
    wl = make()
    out = []
    for tma, stage in ((2, True), (0, False)):
        plan = xx.Plan.from_workload(wl, precision=0)
        plan.set_batch(5, 3)
        plan.set_real_gamma(True)
        plan.set_tma_pass_b(tma)
        plan.set_stage_pass_a(2 if stage else 0)
        ct = gu.dev(wl.c_tgt)
        ex, vx = plan.energy(ct, gu.dev(wl.w_occ), ct, gu.dev(wl.w_tgt), shared=True)
        plan.sync(timeout_s=600.0)
        out.append((vx.cpu().numpy(), float(ex[0].item())))
        plan.close()
    assert gu.rel_max(out[0][0], out[1][0]) <= 1e-6
    assert abs(out[0][1] - out[1][1]) <= 1e-6 * abs(out[1][1])


def test_real_gamma_negative_occupation_sets_the_device_flag(gpu):
    """A negative occupation on the real path (it folds sqrt(w) into the packed slots
    for dE/dmu) is caught on the device: the flag is set, xx_sync reports
    XX_ERR_DEVICE_FLAG and clears it, and the context stays usable."""
    torch, xx = gpu
    wl = synth.real_tiny_cubic()
    w_bad = wl.w_tgt.copy()
    w_bad[0, 1] = -0.5
    plan = xx.Plan.from_workload(wl, precision=1)
    plan.set_real_gamma(True)
    ct = gu.dev(wl.c_tgt)
    plan.backward(ct, gu.dev(w_bad), grad_ex=1.0, want_dc=False)
    with pytest.raises(xx.XXError) as ei:
        plan.sync(timeout_s=120.0)
    assert ei.value.status == -6
    _, dmu = plan.backward(ct, gu.dev(wl.w_tgt), grad_ex=1.0, want_dc=False)
    plan.sync(timeout_s=120.0)
    assert np.isfinite(float(dmu.item()))
    plan.close()
