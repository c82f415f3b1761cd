"""Pins of the oracle's upsampling step on its own (Section 2: the coarse
optimum is doubled and f is evaluated at full resolution for the 3x3
neighbourhood, the minimum kept): numpy brute force over D with exact
fractions on small images, planted noiseless shifts, agreement with the
oracle's full search, and the rejected-coarse contract."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1506_06039_gb300 import synth

INT32_MIN = np.iinfo(np.int32).min


def brute_refine(a, b, sc, tc):
    m, n = b.shape
    best = None
    for u in (-1, 0, 1):
        for v in (-1, 0, 1):
            s, t = 2 * sc + u, 2 * tc + v
            i0, i1, j0, j1 = max(0, -s), min(m, m - s), max(0, -t), min(n, n - t)
            d = a[i0 + s:i1 + s, j0 + t:j1 + t].astype(np.int64) - b[i0:i1, j0:j1].astype(np.int64)
            key = (Fraction(int((d * d).sum()), (i1 - i0) * (j1 - j0)), abs(s) + abs(t), s, t)
            best = key if best is None or key < best else best
    return best


@pytest.mark.parametrize("m,n", [(9, 12), (16, 8), (13, 10)])
def test_refine_matches_brute_force(m, n):
    rng = np.random.default_rng(m * 31 + n)
    b = rng.integers(0, 65536, (m, n)).astype(np.uint16)
    frames = rng.integers(0, 65536, (40, m, n)).astype(np.uint16)
    frames[:8] = b  # some ties (identical frames: f = 0 at (0, 0) for coarse (0, 0))
    hs, ht = (m - 2) // 2, (n - 2) // 2
    coarse = np.stack([rng.integers(-hs, hs + 1, 40), rng.integers(-ht, ht + 1, 40)], 1).astype(np.int32)
    coarse[0] = (hs, -ht)   # candidates out to the frame's last rows and columns
    coarse[1] = (-hs, ht)
    coarse[2:8] = 0
    shifts, ffinal = oracle.refine(frames, b, coarse)
    for f in range(40):
        fr, _, s, t = brute_refine(frames[f], b, int(coarse[f, 0]), int(coarse[f, 1]))
        assert (shifts[f, 0], shifts[f, 1]) == (s, t), f
        assert ffinal[f] == float(fr)


@pytest.mark.parametrize("s0,t0", [(7, -5), (-13, 3), (1, 1), (0, -9), (4, 6)])
def test_refine_recovers_planted_shift(s0, t0):
    m, n = 96, 80
    st = synth.make_stack_np(m, n, 1, 20, 0, seed=700 + s0, template="clean", noise=False)
    b = st.template
    a = np.full((m, n), 100, np.uint16)
    a[max(0, s0):min(m, m + s0), max(0, t0):min(n, n + t0)] = \
        b[max(0, -s0):min(m, m - s0), max(0, -t0):min(n, n - t0)]
    # any coarse whose 3x3 neighbourhood holds the shift: round half away or toward
    for sc in {int(np.floor(s0 / 2)), int(np.ceil(s0 / 2))}:
        for tc in {int(np.floor(t0 / 2)), int(np.ceil(t0 / 2))}:
            shifts, ffinal = oracle.refine(a[None], b, np.array([[sc, tc]], np.int32))
            assert tuple(shifts[0]) == (s0, t0) and ffinal[0] == 0.0


def test_refine_agrees_with_full_search():
    st = synth.make_stack_np(288, 272, 6, 60, 20, seed=99, template="clean")
    r = oracle.align(st.frames, st.template, 8, levels=1)
    shifts, ffinal = oracle.refine(st.frames, st.template, r["coarse"])
    assert np.array_equal(shifts, r["shifts"]) and np.array_equal(ffinal, r["ffinal"])


def test_refine_rejects_coarse_without_overlap():
    m, n = 20, 16
    rng = np.random.default_rng(0)
    b = rng.integers(0, 100, (m, n)).astype(np.uint16)
    frames = rng.integers(0, 100, (4, m, n)).astype(np.uint16)
    coarse = np.array([[10, 0], [0, 8], [-10, 0], [2 ** 30, 1]], np.int32)  # |2 sc| + 1 >= m or |2 tc| + 1 >= n
    shifts, ffinal = oracle.refine(frames, b, coarse)
    assert np.all(shifts == INT32_MIN) and np.all(np.isnan(ffinal))
    ok, _ = oracle.refine(frames[:1], b, np.array([[9, -7]], np.int32))  # the extreme valid coarse shift
    assert ok[0, 0] != INT32_MIN
