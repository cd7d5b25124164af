"""The oracle reproduces its stored fixture (tests/golden/, written by make_golden.py)."""
import json
import os

import numpy as np

from paper_1111_0716_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def test_tiny_cubic_fixture(oracle_mod):
    with open(os.path.join(HERE, "golden", "tiny_cubic_24.json")) as f:
        fx = json.load(f)
    wl = synth.tiny_cubic()
    assert wl.name == fx["workload"]
    vx = oracle_mod.apply(wl)
    e, _ = oracle_mod.energy_from_vx(wl, vx)
    assert abs(e - fx["E_x"]) <= 1e-12 * abs(fx["E_x"])
    for k, a, g, re, im in fx["vx_samples"]:
        assert abs(vx[k, a, g] - (re + 1j * im)) <= 1e-12 * fx["vx_max_abs"]
    assert abs(oracle_mod.pair_sum(wl, which=1) - fx["dE_dmu"]) <= 1e-12 * abs(fx["dE_dmu"])
