"""Strain derivative of E_x (xx_strain_derivative) against Richardson-extrapolated
central differences of the FP64 oracle's E_x with strained lattices
a_i -> a_i (I + eps) at fixed plane-wave coefficients."""
import numpy as np
import pytest

from paper_1111_0716_gb300 import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    return gu.need_gpu()


def rhombo16(kernel):
    return synth.make_workload("rh16", synth.rhombohedral_lattice(6.5, 65.0), (24,) * 3,
                               synth.monkhorst_pack(2), 2.2, 3, 3, [1.0, 0.6, 0.2], 5,
                               kernel=kernel)


def oracle_fd(oracle_mod, wl, al, be, h=1e-4):
    E = np.zeros((3, 3))
    E[al, be] = 1.0

    def e(s):
        return oracle_mod.energy(wl.replace(lattice=wl.lattice @ (np.eye(3) + s * E)))

    def cd(s):
        return (e(s) - e(-s)) / (2 * s)
    return (4 * cd(h) - cd(2 * h)) / 3


def gpu_strain(xx, wl, prec):
    plan = xx.Plan.from_workload(wl, precision=prec)
    c = gu.dev(wl.c_tgt)
    d, e = plan.strain_derivative(c, gu.dev(wl.w_tgt))
    plan.sync(timeout_s=600.0)
    out = d.cpu().numpy(), float(e.item())
    plan.close()
    return out


@pytest.mark.parametrize("kernel", [synth.KERNEL_HSE, synth.KERNEL_COULOMB])
def test_strain_derivative_matches_finite_differences(gpu, oracle_mod, kernel):
    torch, xx = gpu
    wl = rhombo16(kernel)
    d64, e64 = gpu_strain(xx, wl, 1)
    e_ref = oracle_mod.energy(wl)
    assert abs(e64 - e_ref) <= 1e-11 * abs(e_ref)
    assert np.abs(d64 - d64.T).max() <= 1e-13 * np.abs(d64).max()
    scale = np.abs(d64).max()
    w = "rhombo 16^3 strain " + ("screened" if kernel == synth.KERNEL_HSE else "Coulomb")
    for al, be in [(0, 0), (1, 1), (2, 2), (1, 2), (0, 1)]:
        fd = oracle_fd(oracle_mod, wl, al, be)
        assert gu.record(w, 1, "dE/deps_%d%d vs oracle FD" % (al, be), abs(d64[al, be] - fd) / scale,
                         1e-8) <= 1e-8
    d32, e32 = gpu_strain(xx, wl, 0)
    assert gu.record(w, 0, "dE/deps max|d32-d64|/max|d64|", np.abs(d32 - d64).max() / scale,
                     gu.FP32_TOL) <= gu.FP32_TOL
    assert abs(e32 - e64) <= gu.FP32_TOL * abs(e64)


@pytest.mark.parametrize("make", [synth.tiny_cubic, lambda: rhombo16(synth.KERNEL_HSE)])
def test_strain_derivative_pair_symmetry(gpu, make):
    """The pair symmetry (default: k = q tiles, blocks q > k counted twice) and
    transforming every pair agree (FP64)."""
    torch, xx = gpu
    wl = make()
    res = []
    for on in (True, False):
        plan = xx.Plan.from_workload(wl, precision=1)
        plan.set_batch(3, 3)
        plan.set_pair_symmetry(on)
        d, e = plan.strain_derivative(gu.dev(wl.c_tgt), gu.dev(wl.w_tgt))
        res.append((d.cpu().numpy(), float(e.item())))
        plan.close()
    assert np.abs(res[0][0] - res[1][0]).max() <= 1e-12 * np.abs(res[1][0]).max()
    assert abs(res[0][1] - res[1][1]) <= 1e-12 * abs(res[1][1])
