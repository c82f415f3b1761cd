"""The golden fixtures (tests/golden, written by make_golden.py from the
oracle) pinned on the CPU: the worked example against exact integer brute
force of Section 2's definition of f, the planted stack against the
generator's planted shifts; and the oracle still reproduces both."""
import os
from fractions import Fraction

import numpy as np

import oracle
from paper_1506_06039_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_worked():
    lines = [l.split() for l in open(os.path.join(GOLDEN, "worked_3x8_w2.txt")) if not l.startswith("#")]
    m, n, w = map(int, lines[1])
    b = np.array([list(map(int, r)) for r in lines[3:3 + m]], np.uint16)
    a = np.array([list(map(int, r)) for r in lines[4 + m:4 + 2 * m]], np.uint16)
    rows = [tuple(map(int, r)) for r in lines[5 + 2 * m:]]
    return a, b, w, rows


def load_planted():
    out = {}
    for l in open(os.path.join(GOLDEN, "planted_64x72.txt")):
        if l.startswith("#") or l.startswith("levels"):
            continue
        lv, f, s, t, fb, ff = l.split()
        out.setdefault(int(lv), []).append((int(f), int(s), int(t), float(fb), float(ff)))
    return out


def planted_stack():
    return synth.make_stack_np(64, 72, 12, 14, 8, seed=640072, template="clean")


def test_worked_example_is_the_definition():
    a, b, w, rows = load_worked()
    m, n = b.shape
    assert len(rows) == (2 * w - 1) ** 2
    for s, t, S, A in rows:
        ss = sum((int(a[i + s][j + t]) - int(b[i][j])) ** 2
                 for i in range(m) for j in range(n) if 0 <= i + s < m and 0 <= j + t < n)
        aa = sum(1 for i in range(m) for j in range(n) if 0 <= i + s < m and 0 <= j + t < n)
        assert (ss, aa) == (S, A)
    # the content moved one column to the right: f is zero at (0, 1) only
    fs = {(s, t): Fraction(S, A) for s, t, S, A in rows}
    assert fs[(0, 1)] == 0 and sum(v == 0 for v in fs.values()) == 1


def test_oracle_reproduces_worked_example():
    a, b, w, rows = load_worked()
    cost = oracle.cost_surface(a[None], b, w, levels=0)[0]
    for s, t, S, A in rows:
        assert cost[s + w - 1, t + w - 1] == S / A


def test_planted_fixture_matches_planted_shifts_and_oracle():
    st = planted_stack()
    gold = load_planted()
    for levels in (0, 1):
        rec = gold[levels]
        shifts = np.array([(s, t) for _, s, t, _, _ in rec])
        # the generator's truth (clean template) wherever the search can reach it:
        # |s|, |t| <= w - 1 without a level, every planted shift (<= 8) with one
        reach = np.all(np.abs(st.shifts) <= (5 if levels == 0 else 8), axis=1)
        assert reach.sum() >= 4
        assert np.array_equal(shifts[reach], st.shifts[reach])
        r = oracle.align(st.frames, st.template, 6, levels=levels)
        assert np.array_equal(r["shifts"], shifts)
        assert np.array_equal(r["fbest"], np.array([fb for *_, fb, _ in rec]))
        assert np.array_equal(r["ffinal"], np.array([ff for *_, ff in rec]))
