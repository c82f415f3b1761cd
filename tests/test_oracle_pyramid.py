"""Pins of the oracle's general pyramid (L downsamplings, Section 2's
"multiplied by two multiple times"; Section 3's three- and four-level
remark) against numpy downsampling with brute-force sums, noiseless planted
shifts and invariances. CPU only."""
import numpy as np
import pytest

import oracle
from paper_1506_06039_gb300 import synth


def box_levels(a, L):
    """Repeated 2x2 sums with numpy reshapes (floor sizes)."""
    x = a.astype(np.int64)
    for _ in range(L):
        m, n = (x.shape[0] // 2) * 2, (x.shape[1] // 2) * 2
        x = x[:m, :n].reshape(m // 2, 2, n // 2, 2).sum(axis=(1, 3))
    return x


def brute_cost(a, b, w):
    m, n = b.shape
    W = 2 * w - 1
    out = np.empty((W, W))
    for s in range(-(w - 1), w):
        for t in range(-(w - 1), w):
            i0, i1, j0, j1 = max(0, -s), min(m, m - s), max(0, -t), min(n, n - t)
            d = a[i0 + s:i1 + s, j0 + t:j1 + t] - b[i0:i1, j0:j1]
            out[s + w - 1, t + w - 1] = (d * d).sum() / ((i1 - i0) * (j1 - j0))
    return out


@pytest.mark.parametrize("m,n,L,w", [(64, 72, 2, 4), (96, 80, 3, 3), (70, 66, 2, 5)])
def test_searched_level_cost_matches_numpy(m, n, L, w):
    rng = np.random.default_rng(m + n + L)
    a = rng.integers(0, 65536, (m, n)).astype(np.uint16)
    b = rng.integers(0, 65536, (m, n)).astype(np.uint16)
    got = oracle.cost_surface(a[None], b, w, levels=L)[0]
    ref = brute_cost(box_levels(a, L), box_levels(b, L), w) / 16.0 ** L
    assert np.allclose(got, ref, rtol=1e-12, atol=0)


def planted(b, s0, t0, fill=100):
    m, n = b.shape
    a = np.full((m, n), fill, np.uint16)
    a[max(0, s0):min(m, m + s0), max(0, t0):min(n, n + t0)] = \
        b[max(0, -s0):min(m, m - s0), max(0, -t0):min(n, n - t0)]
    return a


@pytest.mark.parametrize("L", [2, 3])
def test_planted_multiple_of_the_level_step_is_exact(L):
    # a shift that is a multiple of 2^L moves every level image by a whole
    # number of its pixels: f = 0 there on every level, and the final shift
    # is the planted one.
    m = n = 256
    st = synth.make_stack_np(m, n, 1, 60, 0, seed=70 + L, template="clean", noise=False)
    b = st.template
    step = 2 ** L
    shifts = [(step * 3, -step * 2), (-step * 5, step), (0, step * 4)]
    frames = np.stack([planted(b, s, t) for s, t in shifts])
    r = oracle.align(frames, b, 8, levels=L)
    assert [tuple(x) for x in r["shifts"]] == shifts
    assert np.all(r["ffinal"] == 0.0)
    assert [tuple(x) for x in r["coarse"]] == [(s // step, t // step) for s, t in shifts]


def test_planted_odd_shifts_recovered_through_the_levels():
    m = n = 256
    st = synth.make_stack_np(m, n, 1, 60, 0, seed=91, template="clean", noise=False)
    b = st.template
    # every shift within reach of one level with w = 6: |s|, |t| <= 2 (w - 1) + 1
    shifts = [(7, -5), (-11, 9), (3, 3), (-1, 10)]
    frames = np.stack([planted(b, s, t) for s, t in shifts])
    for L in (1, 2, 3):
        r = oracle.align(frames, b, 6, levels=L)
        assert [tuple(x) for x in r["shifts"]] == shifts, L
        assert np.all(r["ffinal"] == 0.0)


def test_common_offset_does_not_change_the_result():
    m = n = 128
    st = synth.make_stack_np(m, n, 5, 30, 6, seed=5, template="clean")
    r1 = oracle.align(st.frames, st.template, 4, levels=2)
    add = 1000
    r2 = oracle.align((st.frames.astype(np.int32) + add).astype(np.uint16),
                      (st.template.astype(np.int32) + add).astype(np.uint16), 4, levels=2)
    assert np.array_equal(r1["shifts"], r2["shifts"])
    assert np.array_equal(r1["ffinal"], r2["ffinal"])


def test_rejects_too_many_levels():
    a = np.zeros((64, 64), np.uint16)
    with pytest.raises(ValueError):
        oracle.align(a[None], a, 2, levels=5)
    with pytest.raises(ValueError):
        oracle.align(a[None], a, 5, levels=3)  # 8 x 8 searched grid < 2w - 1
