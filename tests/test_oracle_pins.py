"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these tests re-types the oracle's formula. Each checks the oracle
against something else: closed forms (constant and delta images, the overlap
count), invariants (symmetry, common offset), the paper's own FFT recipe
(Section 2: zero-pad a and the 180-degree-rotated template by w, multiply the
fft2's, ifft2) evaluated with numpy.fft, scipy's 2-D correlation, planted
shifts on noiseless frames, designed exact ties, and central finite
differences for the soft-min gradient.
"""
import numpy as np
import pytest
import scipy.signal

import oracle
from paper_1506_06039_gb300 import synth

rng0 = np.random.default_rng(1234)


def shifts(w):
    return [(s, t) for s in range(-(w - 1), w) for t in range(-(w - 1), w)]


# ---- D_{s,t}, Area and the sign convention (Section 2) ----------------------

@pytest.mark.parametrize("m,n,w", [(7, 9, 4), (12, 5, 3), (16, 16, 6)])
def test_overlap_count_closed_form(m, n, w):
    a = np.ones((m, n), np.int32)
    b = np.zeros((m, n), np.int32)
    S = oracle.ssd_all(a, b, w)
    for s, t in shifts(w):
        assert S[s + w - 1, t + w - 1] == (m - abs(s)) * (n - abs(t))
        assert oracle.area(m, n, s, t) == (m - abs(s)) * (n - abs(t))


@pytest.mark.parametrize("p,q", [(0, 0), (3, 5), (8, 1), (8, 9)])
def test_delta_fixes_sign_convention(p, q):
    # a is one bright pixel at (p, q) and b is zero: the sum over D_{s,t} of
    # a[i+s, j+t]^2 sees the pixel exactly when i = p - s is a valid row and
    # j = q - t a valid column.
    m, n, w, v = 9, 10, 5, 7
    a = np.zeros((m, n), np.int32); a[p, q] = v
    b = np.zeros((m, n), np.int32)
    S = oracle.ssd_all(a, b, w)
    for s, t in shifts(w):
        inside = 0 <= p - s < m and 0 <= q - t < n
        assert S[s + w - 1, t + w - 1] == (v * v if inside else 0)
    # The same pixel in the template instead is seen when (p, q) is in D_{s,t}.
    S2 = oracle.ssd_all(b, a, w)
    for s, t in shifts(w):
        inside = 0 <= p + s < m and 0 <= q + t < n
        assert S2[s + w - 1, t + w - 1] == (v * v if inside else 0)


def test_constant_images_closed_form():
    m, n, w, c1, c2 = 11, 13, 5, 40, 17
    a = np.full((m, n), c1, np.uint16)
    b = np.full((m, n), c2, np.uint16)
    cost = oracle.cost_surface(a, b, w, levels=0)[0]
    assert np.all(cost == (c1 - c2) ** 2)
    r = oracle.align(a, b, w, levels=0)
    assert tuple(r["shifts"][0]) == (0, 0)  # every shift ties: smallest |s|+|t|
    assert r["margin"][0] == 0.0


# ---- The margin (f2 - f1) / f1, f2 the smallest f over every other shift ----
# Hand-worked cases with every f written out as a fraction: a wrong
# denominator (f2 instead of f1), f2 taken among the optimum's own ties, or
# the level's unit applied to one of the two values only changes the number.

def test_margin_hand_worked_delta():
    # 3 x 4, w = 2, b = 0, a = 3 at (1, 1): that pixel is inside the a-side of
    # every D_{s,t}, so S = 9 for all nine shifts and f = 9 / Area with
    # Area = (3 - |s|)(4 - |t|): f(0,0) = 9/12, f(0,+-1) = 9/9, f(+-1,0) = 9/8,
    # f(+-1,+-1) = 9/6. Best (0, 0) = 3/4, next 1: margin (1 - 3/4)/(3/4) = 1/3.
    a = np.zeros((3, 4), np.uint16); a[1, 1] = 3
    b = np.zeros((3, 4), np.uint16)
    cost = oracle.cost_surface(a, b, 2, levels=0)[0]
    assert np.array_equal(cost, np.array([[9 / 6, 9 / 8, 9 / 6], [9 / 9, 9 / 12, 9 / 9], [9 / 6, 9 / 8, 9 / 6]]))
    r = oracle.align(a, b, 2, levels=0)
    assert tuple(r["shifts"][0]) == (0, 0) and r["fbest"][0] == 0.75
    assert r["margin"][0] == pytest.approx(1 / 3, rel=1e-15)


def test_margin_hand_worked_template_bump():
    # 3 x 3, w = 2, a = 1 everywhere, b = 3 at (1, 1) and 0 elsewhere: the
    # template pixel (1, 1) is in every D, so S = (Area - 1) * 1 + (1 - 3)^2
    # = Area + 3 and f = 1 + 3 / Area: f(0,0) = 4/3, f at one-axis shifts 3/2,
    # at diagonal shifts 7/4. Margin (3/2 - 4/3) / (4/3) = 1/8.
    a = np.ones((3, 3), np.uint16)
    b = np.zeros((3, 3), np.uint16); b[1, 1] = 3
    r = oracle.align(a, b, 2, levels=0)
    assert tuple(r["shifts"][0]) == (0, 0) and r["fbest"][0] == pytest.approx(4 / 3, rel=1e-15)
    assert r["margin"][0] == pytest.approx(1 / 8, rel=1e-15)


def test_margin_hand_worked_one_level():
    # The delta case at twice the size with one 2x2 level: a 2x2 block of 3s
    # at rows 2-3, columns 2-3 of a 6 x 8 frame sums to 12 at coarse (1, 1),
    # so the searched-grid costs are 144 / Area / 16 in box-mean units, the
    # same fractions as the delta case: fbest 3/4, margin 1/3.
    a = np.zeros((6, 8), np.uint16); a[2:4, 2:4] = 3
    b = np.zeros((6, 8), np.uint16)
    r = oracle.align(a, b, 2, levels=1)
    assert tuple(r["coarse"][0]) == (0, 0) and r["fbest"][0] == 0.75
    assert r["margin"][0] == pytest.approx(1 / 3, rel=1e-15)


def test_margin_best_away_from_centre():
    # b[i][j] = 10 j + 3 i^2 and a the same image moved right by one column
    # (a[i][j] = b[i][j-1], first column 0): f(0, 1) = 0 exactly is the optimum
    # and every other shift has f > 0 (b varies along both axes), so
    # the margin is infinite; with the frame's first column raised from 0 to 5
    # the optimum stays at (0, 1) with S = 0 still (that column is outside
    # D_{0,1}'s a-side), so the margin stays infinite: the margin is taken over
    # the other shifts only, never over the optimum itself.
    m, n = 5, 6
    b = (10 * np.arange(n)[None, :] + 3 * np.arange(m)[:, None] ** 2).astype(np.uint16)
    a = np.zeros((m, n), np.uint16); a[:, 1:] = b[:, :-1]
    for first in (0, 5):
        a[:, 0] = first
        r = oracle.align(a, b, 2, levels=0)
        assert tuple(r["shifts"][0]) == (0, 1) and r["fbest"][0] == 0 and r["margin"][0] == np.inf


# ---- Invariants ---------------------------------------------------------------

def test_identity_gives_zero_shift():
    a = rng0.integers(0, 4000, (20, 24)).astype(np.uint16)
    cost = oracle.cost_surface(a, a, 6, levels=0)[0]
    assert cost[5, 5] == 0.0 and np.all(np.delete(cost.ravel(), 5 * 11 + 5) > 0)
    r = oracle.align(a, a, 6, levels=0)
    assert tuple(r["shifts"][0]) == (0, 0) and r["margin"][0] == np.inf


@pytest.mark.parametrize("s0,t0", [(3, -2), (-4, 4), (0, 1), (-1, -3)])
def test_planted_shift_noiseless(s0, t0):
    m, n, w = 18, 21, 6
    b = rng0.integers(0, 3000, (m, n)).astype(np.uint16)
    a = np.full((m, n), 100, np.uint16)
    for i in range(m):
        for j in range(n):
            if 0 <= i - s0 < m and 0 <= j - t0 < n:
                a[i, j] = b[i - s0, j - t0]
    cost = oracle.cost_surface(a, b, w, levels=0)[0]
    assert cost[s0 + w - 1, t0 + w - 1] == 0.0
    r = oracle.align(a, b, w, levels=0)
    assert tuple(r["shifts"][0]) == (s0, t0)


def test_symmetry_swapping_frame_and_template():
    a = rng0.integers(0, 5000, (15, 17)).astype(np.int32)
    b = rng0.integers(0, 5000, (15, 17)).astype(np.int32)
    w = 6
    S_ab = oracle.ssd_all(a, b, w)
    S_ba = oracle.ssd_all(b, a, w)
    assert np.array_equal(S_ab, S_ba[::-1, ::-1])


def test_common_offset_invariance():
    a = rng0.integers(0, 5000, (14, 19)).astype(np.int32)
    b = rng0.integers(0, 5000, (14, 19)).astype(np.int32)
    assert np.array_equal(oracle.ssd_all(a, b, 5), oracle.ssd_all(a - 777, b - 777, 5))


# ---- The three-sum expansion and the paper's FFT recipe (Section 2) ----------

def _energies(a, b, w):
    m, n = a.shape
    W = 2 * w - 1
    Ea = np.zeros((W, W), np.int64)
    Eb = np.zeros((W, W), np.int64)
    for s, t in shifts(w):
        i0, i1 = max(0, -s), min(m, m - s)
        j0, j1 = max(0, -t), min(n, n - t)
        Eb[s + w - 1, t + w - 1] = int((b[i0:i1, j0:j1].astype(np.int64) ** 2).sum())
        Ea[s + w - 1, t + w - 1] = int((a[i0 + s:i1 + s, j0 + t:j1 + t].astype(np.int64) ** 2).sum())
    return Ea, Eb


def test_expansion_with_scipy_correlation():
    m, n, w = 16, 13, 6
    a = rng0.integers(0, 3000, (m, n)).astype(np.int64)
    b = rng0.integers(0, 3000, (m, n)).astype(np.int64)
    Ea, Eb = _energies(a, b, w)
    c = scipy.signal.correlate2d(a, b, mode="full")  # c[s+m-1, t+n-1] = sum a[i+s,j+t] b[i,j]
    h = c[m - 1 - (w - 1):m + w - 1, n - 1 - (w - 1):n + w - 1]
    assert np.array_equal(oracle.ssd_all(a, b, w), Ea + Eb - 2 * h)


@pytest.mark.parametrize("m,n,w", [(12, 12, 4), (16, 10, 5), (9, 14, 3)])
def test_paper_fft_recipe(m, n, w):
    # fft2 of [[a, zeros(m, w)]; zeros(w, n + w)] and of the same padding of
    # the 180-degree rotation of b; the ifft2 of their product holds
    # h[s, t] at (s + m - 1, t + n - 1).
    a = rng0.integers(0, 2000, (m, n)).astype(np.float64)
    b = rng0.integers(0, 2000, (m, n)).astype(np.float64)
    pad = lambda x: np.pad(x, ((0, w), (0, w)))
    h_full = np.real(np.fft.ifft2(np.fft.fft2(pad(a)) * np.fft.fft2(pad(b[::-1, ::-1]))))
    Ea, Eb = _energies(a.astype(np.int64), b.astype(np.int64), w)
    W = 2 * w - 1
    h = np.zeros((W, W))
    for s, t in shifts(w):
        h[s + w - 1, t + w - 1] = h_full[s + m - 1, t + n - 1]
    S_fft = Ea + Eb - 2 * np.rint(h).astype(np.int64)
    assert np.array_equal(oracle.ssd_all(a.astype(np.int32), b.astype(np.int32), w), S_fft)


# ---- Downsampling --------------------------------------------------------------

def test_downsample_closed_forms():
    a = np.full((8, 6), 1000, np.uint16)
    assert np.all(oracle.downsample(a) == 4000)
    z = np.zeros((8, 6), np.uint16)
    z[5, 2] = 65535
    d = oracle.downsample(z)
    assert d[2, 1] == 65535 and d.sum() == 65535
    r = rng0.integers(0, 65536, (10, 12)).astype(np.uint16)
    assert oracle.downsample(r).sum() == r.astype(np.int64).sum()
    assert oracle.downsample(np.full((4, 4), 65535, np.uint16)).max() == 4 * 65535
    assert oracle.levels(256, 256) == 0 and oracle.levels(257, 100) == 1 and oracle.levels(512, 512) == 1


# ---- Tie-break (the paper is silent; smallest |s|+|t|, then s, then t) -------

def test_tiebreak_rows():
    m, n, k = 12, 12, 50
    i = np.arange(m)[:, None] * np.ones((1, n), int)
    b = ((i % 2) * k).astype(np.uint16)
    a = (((i + 1) % 2) * k).astype(np.uint16)
    r = oracle.align(a, b, 4, levels=0)
    assert tuple(r["shifts"][0]) == (-1, 0) and r["fbest"][0] == 0 and r["margin"][0] == 0


def test_tiebreak_columns():
    m, n, k = 12, 12, 50
    j = np.ones((m, 1), int) * np.arange(n)[None, :]
    b = ((j % 2) * k).astype(np.uint16)
    a = (((j + 1) % 2) * k).astype(np.uint16)
    r = oracle.align(a, b, 4, levels=0)
    assert tuple(r["shifts"][0]) == (0, -1)


def test_tiebreak_checkerboard():
    m, n, k = 10, 10, 9
    i, j = np.indices((m, n))
    b = (((i + j) % 2) * k).astype(np.uint16)
    a = (((i + j + 1) % 2) * k).astype(np.uint16)
    r = oracle.align(a, b, 3, levels=0)
    assert tuple(r["shifts"][0]) == (-1, 0)


# ---- Upsampling jitter on a planted full-resolution shift ---------------------

@pytest.mark.parametrize("s0,t0", [(5, -3), (-7, 2), (4, 4), (1, -1)])
def test_jitter_recovers_odd_full_resolution_shift(s0, t0):
    m = n = 264  # > 256: one 2x2 level, 132x132 coarse grid
    st = synth.make_stack_np(m, n, 1, 30, 0, seed=99 + s0, template="clean", noise=False)
    b = st.template
    a = np.full((m, n), 100, np.uint16)
    a[max(0, s0):min(m, m + s0), max(0, t0):min(n, n + t0)] = \
        b[max(0, -s0):min(m, m - s0), max(0, -t0):min(n, n - t0)]
    r = oracle.align(a, b, 6)
    assert tuple(r["shifts"][0]) == (s0, t0)
    assert r["ffinal"][0] == 0.0
    assert abs(2 * r["coarse"][0, 0] - s0) <= 1 and abs(2 * r["coarse"][0, 1] - t0) <= 1


def test_cost_surface_units_and_levels():
    # Box-mean units: the coarse 4-sum cost divided by 16; with no level the
    # cost is the plain f.
    st = synth.make_stack_np(264, 264, 1, 20, 3, seed=5, template="clean")
    c1, S = oracle.cost_surface(st.frames, st.template, 4, with_sums=True)
    ac, bc = oracle.downsample(st.frames[0]), oracle.downsample(st.template)
    assert np.array_equal(S[0], oracle.ssd_all(ac, bc, 4))
    for s, t in shifts(4):
        assert c1[0, s + 3, t + 3] == S[0, s + 3, t + 3] / oracle.area(132, 132, s, t) / 16.0


def test_align_matches_planted_shifts_on_small_stack():
    st = synth.make_stack_np(64, 64, 12, 12, 5, seed=7, template="clean")
    r = oracle.align(st.frames, st.template, 8, levels=0, nthreads=2)
    assert np.array_equal(r["shifts"], st.shifts)


# ---- Soft-min form (not in the paper): loss and gradient ---------------------

def test_softmin_single_shift_closed_form():
    m, n = 6, 7
    a = rng0.uniform(0, 100, (m, n))
    b = rng0.uniform(0, 100, (m, n))
    L, lf, gb, ga = oracle.softmin_loss(a, b, 1, [3.0], grad_template=True, grad_frames=True)
    f00 = ((a - b) ** 2).mean()
    assert L == pytest.approx(f00, rel=1e-13)
    np.testing.assert_allclose(gb, -2 * (a - b) / (m * n), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(ga[0], 2 * (a - b) / (m * n), rtol=1e-12, atol=1e-14)


def test_softmin_equal_costs_closed_form():
    m, n, w, tau = 8, 9, 3, 0.7
    a = np.full((m, n), 5.0)
    b = np.full((m, n), 2.0)
    L, *_ = oracle.softmin_loss(a, b, w, [tau])
    assert L == pytest.approx(9.0 - tau * np.log((2 * w - 1) ** 2), rel=1e-13)


def test_softmin_small_tau_tends_to_min():
    a = rng0.uniform(0, 100, (10, 10))
    b = rng0.uniform(0, 100, (10, 10))
    cost = oracle.cost_f64(a, b, 3)
    L, *_ = oracle.softmin_loss(a, b, 3, [1e-6])
    assert L == pytest.approx(cost.min(), rel=1e-9)


def test_median_odd_count():
    v = rng0.normal(size=961)
    assert oracle.median(v) == np.median(v)


def test_cost_f64_agrees_with_exact_integer_cost():
    a = rng0.integers(0, 9000, (13, 15)).astype(np.uint16)
    b = rng0.integers(0, 9000, (13, 15)).astype(np.uint16)
    exact = oracle.cost_surface(a, b, 5, levels=0)[0]
    np.testing.assert_allclose(oracle.cost_f64(a, b, 5), exact, rtol=1e-14)


@pytest.mark.parametrize("which", ["template", "frames"])
def test_softmin_gradient_central_differences(which):
    rng = np.random.default_rng(11)
    T, m, n, w = 2, 7, 8, 3
    a = rng.uniform(50, 500, (T, m, n))
    b = rng.uniform(50, 500, (m, n))
    tau = oracle.softmin_tau(a, b, w)
    _, _, gb, ga = oracle.softmin_loss(a, b, w, tau, grad_template=True, grad_frames=True)
    eps = 1e-3
    for _ in range(12):
        i, j = rng.integers(0, m), rng.integers(0, n)
        if which == "template":
            bp, bm = b.copy(), b.copy()
            bp[i, j] += eps; bm[i, j] -= eps
            fd = (oracle.softmin_loss(a, bp, w, tau)[0] - oracle.softmin_loss(a, bm, w, tau)[0]) / (2 * eps)
            assert gb[i, j] == pytest.approx(fd, rel=1e-6, abs=1e-9)
        else:
            f = rng.integers(0, T)
            ap, am = a.copy(), a.copy()
            ap[f, i, j] += eps; am[f, i, j] -= eps
            fd = (oracle.softmin_loss(ap, b, w, tau)[0] - oracle.softmin_loss(am, b, w, tau)[0]) / (2 * eps)
            assert ga[f, i, j] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_softmin_zero_tau_is_the_min():
    # tau = 0: the soft-min is the min, its weight split over the minimisers.
    a = np.full((6, 8), 4.0)
    b = np.full((6, 8), 4.0)
    L, lf, gb, _ = oracle.softmin_loss(a, b, 2, [0.0], grad_template=True)
    assert L == 0.0 and np.all(gb == 0.0)
