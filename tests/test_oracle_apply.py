"""Pins of the oracle's correction step (applying the found shifts, Section 2's
"motion corrected" output) against hand-worked values, an undone planted
shift, identities and the fill rule. CPU only."""
import numpy as np

import oracle


def test_worked_example_by_hand():
    # frame 0: 0..11 as 3x4, frame 1: 12..23; shifts (0,0) and (1,-1), fill 7.
    a = np.arange(24, dtype=np.uint16).reshape(2, 3, 4)
    c, mu = oracle.apply_shifts(a, [[0, 0], [1, -1]], fill=7)
    # frame 1 corrected[i][j] = a1[i+1][j-1]: row 0 <- a1 row 1 (16..19) moved
    # right by one column, row 1 <- a1 row 2 (20..23), row 2 <- outside.
    assert c[0].tolist() == [[0, 1, 2, 3], [4, 5, 6, 7], [8, 9, 10, 11]]
    assert c[1].tolist() == [[7, 16, 17, 18], [7, 20, 21, 22], [7, 7, 7, 7]]
    # mean over the frames whose source pixel is inside: column 0 and row 2
    # only have frame 0; elsewhere (x + y) / 2.
    assert mu.tolist() == [[0.0, 8.5, 9.5, 10.5], [4.0, 12.5, 13.5, 14.5], [8.0, 9.0, 10.0, 11.0]]


def test_undoes_a_planted_shift():
    rng = np.random.default_rng(11)
    m, n = 37, 24
    x = rng.integers(0, 65536, (m, n)).astype(np.uint16)
    for s, t in [(3, -5), (-7, 2), (0, 11), (-36, 23)]:
        # content moved by +(s, t): frame[i][j] = x[i-s][j-t], background 100
        frame = np.full((m, n), 100, np.uint16)
        for i in range(m):
            for j in range(n):
                if 0 <= i - s < m and 0 <= j - t < n:
                    frame[i, j] = x[i - s, j - t]
        c, mu = oracle.apply_shifts(frame[None], [[s, t]], fill=9)
        for i in range(m):
            for j in range(n):
                inside = 0 <= i + s < m and 0 <= j + t < n
                assert c[0, i, j] == (x[i, j] if inside else 9)
                assert mu[i, j] == (float(x[i, j]) if inside else 9.0)


def test_zero_shifts_are_the_identity_and_numpy_mean():
    rng = np.random.default_rng(12)
    a = rng.integers(0, 65536, (9, 16, 8)).astype(np.uint16)
    c, mu = oracle.apply_shifts(a, np.zeros((9, 2), np.int32), fill=3)
    assert np.array_equal(c, a)
    assert np.array_equal(mu, a.astype(np.float64).sum(0) / 9.0)


def test_shift_past_the_frame_is_all_fill():
    a = np.full((2, 5, 8), 1234, np.uint16)
    c, mu = oracle.apply_shifts(a, [[5, 0], [0, -8]], fill=42)
    assert np.all(c == 42) and np.all(mu == 42.0)


def test_mean_counts_only_covering_frames():
    # three constant frames 10, 20, 30 shifted by 0, +1, +2 rows: row 0 is
    # covered by all three, row m-2 by two, row m-1 by one.
    m, n = 6, 8
    a = np.stack([np.full((m, n), v, np.uint16) for v in (10, 20, 30)])
    _, mu = oracle.apply_shifts(a, [[0, 0], [1, 0], [2, 0]], fill=0)
    assert np.all(mu[: m - 2] == 20.0)
    assert np.all(mu[m - 2] == 15.0)
    assert np.all(mu[m - 1] == 10.0)
