"""Writes the stored expected values under tests/golden/ from the FP64 oracle only.

Run from the repository root:  python tests/golden/make_golden.py
Each fixture records the seeded workload it came from; the values are the
oracle's, which the pins in tests/test_oracle_pins.py tie to mathematics.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_1111_0716_gb300 import synth  # noqa: E402


def fixture(wl, sample):
    vx = oracle.apply(wl)
    e_re, e_im = oracle.energy_from_vx(wl, vx)
    return {
        "workload": wl.name, "seed": wl.seed, "grid": list(wl.grid), "nk": wl.nk,
        "n_occ": wl.n_occ, "n_tgt": wl.n_tgt, "kernel": wl.kernel, "mu": wl.mu,
        "E_x": e_re, "E_x_imag": e_im,
        "dE_dmu": oracle.pair_sum(wl, which=1) if wl.kernel == synth.KERNEL_HSE else None,
        "vx_samples": [[k, a, g, float(vx[k, a, g].real), float(vx[k, a, g].imag)]
                       for (k, a, g) in sample],
        "vx_max_abs": float(np.abs(vx).max()),
    }


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    wl = synth.tiny_cubic()
    out = fixture(wl, [(0, 0, 0), (0, 3, 100), (0, 7, 484)])
    with open(os.path.join(here, "tiny_cubic_24.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
