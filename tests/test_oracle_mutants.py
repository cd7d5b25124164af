"""The oracle's pins reject broken copies of the oracle.

Each case below plants one plausible mistake in a copy of ``oracle/xx_oracle.c``
(a flipped sign, a dropped factor, a conjugate on the wrong operand, a
transposed index), compiles the copy on the CPU, and runs the pin suite
(``tests/test_oracle_pins.py``) against it through ``XX_ORACLE_LIB``.  The pins
must fail for every planted mistake: a mistake that no pin sees would mean the
oracle could carry it unnoticed.  The committed oracle itself is never changed.
"""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "xx_oracle.c")

# (name, exact text in xx_oracle.c, its replacement).  Each text occurs exactly once.
MUTANTS = [
    # FFT
    ("fft_twiddle_sign",
     "double ang = sign * 2.0 * M_PI",
     "double ang = -sign * 2.0 * M_PI"),
    ("fft_twiddle_index",
     "long e = ((long)r * kk) % n;",
     "long e = ((long)r * k) % n;"),
    # reciprocal lattice and kernel
    ("reciprocal_transposed",
     "g[c] += md[i] * B[3 * i + c];",
     "g[c] += md[i] * B[3 * c + i];"),
    ("kernel_screening_dropped",
     "return 4.0 * M_PI / g2 * (-expm1(-g2 / (4.0 * mu * mu)));",
     "return 4.0 * M_PI / g2;"),
    ("kernel_g0_limit_dropped",
     "if (is_zero) return M_PI / (mu * mu);",
     "if (is_zero) return 0.0;"),
    ("kernel_dmu_sign",
     "return -2.0 * M_PI / (mu * mu * mu) * exp(-g2 / (4.0 * mu * mu));",
     "return 2.0 * M_PI / (mu * mu * mu) * exp(-g2 / (4.0 * mu * mu));"),
    ("kernel_dmu_exponent",
     "return -2.0 * M_PI / (mu * mu * mu) * exp(-g2 / (4.0 * mu * mu));",
     "return -2.0 * M_PI / (mu * mu * mu) * exp(-g2 / (2.0 * mu * mu));"),
    # sphere <-> grid
    ("sphere_to_grid_scale_dropped",
     "double s = 1.0 / sqrt(omega);",
     "double s = 1.0;"),
    ("grid_to_sphere_direction",
     "oracle_fft3d(f, grid[0], grid[1], grid[2], -1);",
     "oracle_fft3d(f, grid[0], grid[1], grid[2], +1);"),
    ("grid_to_sphere_scale",
     "double s = sqrt(omega) / (double)ntot;",
     "double s = 1.0 / (sqrt(omega) * (double)ntot);"),
    # the operator's loops
    ("codensity_conjugates_target",
     "for (long p = 0; p < ntot; ++p) rho[p] = conj(uj[p]) * ua[p];",
     "for (long p = 0; p < ntot; ++p) rho[p] = uj[p] * conj(ua[p]);"),
    ("accumulate_with_conj_occupied",
     "acct[p] += f * uj[p] * rho[p];",
     "acct[p] += f * conj(uj[p]) * rho[p];"),
    ("accumulate_with_target",
     "acct[p] += f * uj[p] * rho[p];",
     "acct[p] += f * ua[p] * rho[p];"),
    ("kernel_normalisation_dropped",
     "for (long p = 0; p < ntot; ++p) rho[p] *= v[p] / (double)ntot;",
     "for (long p = 0; p < ntot; ++p) rho[p] *= v[p];"),
    ("k_minus_q_reversed",
     "u_occ + ntot * j);\n"
     "            double d[3] = {kfrac[3 * k] - kfrac[3 * q], kfrac[3 * k + 1] - kfrac[3 * q + 1],\n"
     "                           kfrac[3 * k + 2] - kfrac[3 * q + 2]};",
     "u_occ + ntot * j);\n"
     "            double d[3] = {kfrac[3 * q] - kfrac[3 * k], kfrac[3 * q + 1] - kfrac[3 * k + 1],\n"
     "                           kfrac[3 * q + 2] - kfrac[3 * k + 2]};"),
    ("occupation_dropped",
     "const double f = -wq / (double)nk;",
     "const double f = -1.0 / (double)nk;"),
    ("k_mesh_weight_dropped",
     "const double f = -wq / (double)nk;",
     "const double f = -wq;"),
    ("operator_sign",
     "const double f = -wq / (double)nk;",
     "const double f = wq / (double)nk;"),
    # reductions
    ("energy_spin_factor_dropped",
     "e *= 0.5 * ORACLE_SPIN_FACTOR / (double)nk;",
     "e *= 0.5 / (double)nk;"),
    ("energy_conjugate_dropped",
     "for (int g = 0; g < npw[k]; ++g) dot += conj(c[g]) * y[g];",
     "for (int g = 0; g < npw[k]; ++g) dot += c[g] * y[g];"),
    ("pair_sum_volume_dropped",
     "return -0.5 * ORACLE_SPIN_FACTOR * omega / ((double)nk * (double)nk) * total;",
     "return -0.5 * ORACLE_SPIN_FACTOR / ((double)nk * (double)nk) * total;"),
    ("pair_sum_target_weight_dropped",
     "total += wa * wj * s;",
     "total += wj * s;"),
]


def test_each_planted_text_occurs_once():
    src = open(SRC).read()
    names = [m[0] for m in MUTANTS]
    assert len(names) == len(set(names))
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, name
        assert old != new, name


@pytest.fixture(scope="module")
def source():
    return open(SRC).read()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_the_planted_mistake(tmp_path, source, name, old, new):
    c_file = tmp_path / (name + ".c")
    so_file = tmp_path / ("lib" + name + ".so")
    c_file.write_text(source.replace(old, new))
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                           "-o", str(so_file), str(c_file), "-lm"])
    env = dict(os.environ, XX_ORACLE_LIB=str(so_file))
    out = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q",
                          "-p", "no:cacheprovider", "-W", "ignore"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    # exit status 1: some test failed (0 would mean every pin passed with the mistake in)
    assert out.returncode == 1, (name, out.returncode, out.stdout[-3000:])
    assert re.search(r"^FAILED tests/test_oracle_pins.py::", out.stdout, re.M), out.stdout[-3000:]
