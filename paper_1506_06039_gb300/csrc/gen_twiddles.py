"""Writes twiddles.cuh: the roots of unity used inside the register codelets.

For every composite codelet size R the header holds omega_R^k = exp(-2 pi i k / R),
k = 0..R-1, computed in FP64 from math.cos / math.sin of the exact rational
angle and rounded once to FP32. Run: python gen_twiddles.py (writes beside it).
"""
import math
import os

SIZES = [6, 8, 9, 10, 12, 15, 16, 18, 20, 24, 25, 27, 30, 32, 36]


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "twiddles.cuh")
    lines = [
        "// Generated by gen_twiddles.py: omega_R^k = exp(-2 pi i k / R) for the",
        "// composite register codelets, FP64 cos/sin rounded once to FP32.",
        "#pragma once",
        "#include <cuda_runtime.h>",
        "namespace moco {",
    ]
    for R in SIZES:
        vals = []
        for k in range(R):
            ang = 2.0 * math.pi * k / R
            c, s = math.cos(ang), -math.sin(ang)
            if k * 4 % R == 0:  # exact quarter turns
                c, s = [(1.0, 0.0), (0.0, -1.0), (-1.0, 0.0), (0.0, 1.0)][k * 4 // R]
            vals.append("{%.17ef, %.17ef}" % (c, s))
        lines.append("static __constant__ float2 c_tw%d[%d] = {%s};" % (R, R, ", ".join(vals)))
    lines.append("template <int R> struct Tw;")
    for R in SIZES:
        lines.append("template <> struct Tw<%d> { __device__ static float2 get(int k) { return c_tw%d[k]; } };" % (R, R))
    lines.append("}  // namespace moco")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
