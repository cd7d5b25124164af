"""The FFT lengths 36 (6 x 6), 54 (6 x 9) and 108 (6 x 18), each through every
pass (sphere <-> grid, the three band-pair passes, the role-swapped pass C of
the pair symmetry), against the FP64 oracle in both precisions; one cell mixes
two of them (54 x 54 x 108)."""
import math

import numpy as np
import pytest

from paper_1111_0716_gb300 import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    return gu.need_gpu()


def cell36():
    return synth.make_workload("cubic-36^3-MP2", synth.cubic_lattice(15.0), (36,) * 3,
                               synth.monkhorst_pack(2), math.pi, 4, 6, [1.0, 1.0, 0.6, 0.3], 81)


def cell54():
    return synth.make_workload("rhombo-54^3", synth.rhombohedral_lattice(20.0, 62.0), (54,) * 3,
                               np.zeros((1, 3)), 2.0, 5, 6, [1.0] * 5, 82)


def cell108():
    return synth.make_workload("cubic-108^3", synth.cubic_lattice(20.0), (108,) * 3,
                               np.zeros((1, 3)), 0.5 * math.pi, 4, 5, [1.0, 1.0, 1.0, 0.5], 83)


def cell54x108():
    return synth.make_workload("tetra-54x54x108", np.diag([12.0, 12.0, 24.0]), (54, 54, 108),
                               np.zeros((1, 3)), 0.8 * math.pi, 4, 4, [1.0] * 4, 84)


CELLS = {"36": cell36, "54": cell54, "108": cell108, "54x54x108": cell54x108}


@pytest.mark.parametrize("name", sorted(CELLS))
@pytest.mark.parametrize("prec,tol", [(0, gu.FP32_TOL), (1, gu.FP64_TOL)])
def test_new_lengths_match_oracle(gpu, oracle_mod, name, prec, tol):
    wl = CELLS[name]()
    assert np.all(4 * wl.n_max() + 1 <= np.array(wl.grid))
    ref = oracle_mod.apply(wl)
    e_ref, _ = oracle_mod.energy_from_vx(wl, ref)
    vx, (e, _), _ = gu.run(wl, prec)
    w = "%s (%s)" % (wl.name, "x".join(map(str, wl.grid)))
    assert gu.record(w, prec, "max|dVx|/max|Vx|", gu.rel_max(vx, ref), tol) <= tol
    assert gu.record(w, prec, "|dE_x|/|E_x|", gu.rel_err(e, e_ref), tol) <= tol
