"""Writes xx_roots.cuh: cos/sin(2 pi m / R) for the in-register composite DFTs.

Run from this directory:  python gen_roots.py
The values are evaluated with 40 significant digits (mpmath) and then rounded
to the nearest double; the CUDA code rounds them to float for the FP32 path.
"""
import mpmath

mpmath.mp.dps = 40


def _c(R, m):
    return float(mpmath.cos(2 * mpmath.pi * m / R))


def _s(R, m):
    return float(mpmath.sin(2 * mpmath.pi * m / R))

RADICES = (6, 9, 10, 12, 16, 18)


def main():
    lines = ["// Generated by gen_roots.py: unit roots exp(2 pi i m / R) for composite",
             "// in-register DFT lengths.  Do not edit by hand.",
             "#pragma once", "",
             "__device__ __forceinline__ constexpr double xx_root_cos(int R, int m) {",
             "  return"]
    body_c, body_s = [], []
    for R in RADICES:
        for m in range(R):
            body_c.append("    (R == %d && m == %d) ? %r :" % (R, m, _c(R, m)))
            body_s.append("    (R == %d && m == %d) ? %r :" % (R, m, _s(R, m)))
    lines += body_c + ["    0.0;", "}", "",
                       "__device__ __forceinline__ constexpr double xx_root_sin(int R, int m) {",
                       "  return"] + body_s + ["    0.0;", "}", ""]
    with open("xx_roots.cuh", "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
