"""Writes the golden fixtures of this directory from the oracle alone.

    python tests/golden/make_golden.py

worked_3x8_w2.txt : Section 2's cost f_{s,t} for a 3 x 8 template and a
    frame whose content moved one column to the right (w = 2, nine shifts),
    stored as exact integers S (sum of squared differences over the overlap
    D_st) and A (= Area(D_st)), f = S / A.
planted_64x72.txt : a seeded 12-frame stack (64 x 72, w = 6, no level and one
    level): the oracle's shifts, best costs and final full-resolution costs.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1506_06039_gb300 import synth  # noqa: E402


def worked():
    b = np.arange(1, 25, dtype=np.uint16).reshape(3, 8)
    a = np.zeros_like(b)
    a[:, 1:] = b[:, :-1]  # content moved by +1 column: a[i][j + 1] = b[i][j]
    w = 2
    cost = oracle.cost_surface(a[None], b, w, levels=0)[0]
    lines = ["# Section 2, Eq. for f_{s,t}: f = S / A with S the sum over the overlap D_st of",
             "# (a[i+s][j+t] - b[i][j])^2 and A = Area(D_st) = (m - |s|)(n - |t|); shifts |s|,|t| < w.",
             "# Written by make_golden.py from oracle.cost_surface (S = f * A, exact integers here).",
             "m n w", "3 8 %d" % w, "template"]
    lines += [" ".join(str(int(v)) for v in row) for row in b]
    lines.append("frame")
    lines += [" ".join(str(int(v)) for v in row) for row in a]
    lines.append("s t S A")
    for s in range(-(w - 1), w):
        for t in range(-(w - 1), w):
            A = (3 - abs(s)) * (8 - abs(t))
            S = cost[s + w - 1, t + w - 1] * A
            assert abs(S - round(S)) < 1e-9
            lines.append("%d %d %d %d" % (s, t, int(round(S)), A))
    with open(os.path.join(HERE, "worked_3x8_w2.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


def planted():
    st = synth.make_stack_np(64, 72, 12, 14, 8, seed=640072, template="clean")
    lines = ["# Oracle results (Section 2 search; with levels = 1 the 2x2-box level and the",
             "# 3x3 full-resolution jitter) for synth.make_stack_np(64, 72, 12, 14, 8, seed=640072,",
             "# template='clean'), w = 6. Written by make_golden.py from oracle.align.",
             "levels frame s t fbest ffinal"]
    for levels in (0, 1):
        r = oracle.align(st.frames, st.template, 6, levels=levels)
        for f in range(st.frames.shape[0]):
            lines.append("%d %d %d %d %.17g %.17g" % (levels, f, r["shifts"][f, 0], r["shifts"][f, 1],
                                                       r["fbest"][f], r["ffinal"][f]))
    with open(os.path.join(HERE, "planted_64x72.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    worked()
    planted()
