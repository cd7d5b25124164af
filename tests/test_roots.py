"""The compile-time unit roots of the in-register composite DFTs (csrc/xx_roots.cuh).

The table is generated, not typed: regenerating it gives the committed file byte
for byte, and every entry is cos/sin(2 pi m / R) rounded to double (checked
against numpy on the double-rounded angle, whose own error is below 1e-15)."""
import math
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1111_0716_gb300", "csrc")


def table():
    src = open(os.path.join(CSRC, "xx_roots.cuh")).read()
    out = {}
    for fn in ("cos", "sin"):
        body = src[src.index("xx_root_%s" % fn):]
        body = body[:body.index("}")]
        for R, m, v in re.findall(r"\(R == (\d+) && m == (\d+)\) \? ([-0-9.e]+) :", body):
            out[(fn, int(R), int(m))] = float(v)
    return out


def test_every_root_is_the_rounded_unit_root():
    t = table()
    radices = sorted({R for _, R, _ in t})
    assert radices == [6, 9, 10, 12, 16, 18]
    for R in radices:
        for m in range(R):
            ang = 2.0 * math.pi * m / R
            assert abs(t[("cos", R, m)] - np.cos(ang)) <= 1e-15, (R, m)
            assert abs(t[("sin", R, m)] - np.sin(ang)) <= 1e-15, (R, m)
            # symmetries of the unit circle (zeros such as sin(pi) or cos(pi/2) are
            # evaluated at 40 digits, so the table holds 1e-43..1e-41 there, far below
            # any rounding error of the transforms)
            assert abs(t[("cos", R, m)] - t[("cos", R, (R - m) % R)]) <= 1e-40
            assert abs(t[("sin", R, m)] + t[("sin", R, (R - m) % R)]) <= 1e-40


def test_regenerating_gives_the_committed_file(tmp_path):
    pytest.importorskip("mpmath")
    subprocess.check_call([sys.executable, os.path.join(CSRC, "gen_roots.py")], cwd=tmp_path)
    with open(os.path.join(CSRC, "xx_roots.cuh")) as f:
        committed = f.read()
    assert (tmp_path / "xx_roots.cuh").read_text() == committed
