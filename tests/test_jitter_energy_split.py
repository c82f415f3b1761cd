"""The decomposition the full-resolution refinement uses for sum_D a^2 of its
nine candidates, checked on the host against the direct sum: each thread of
a band sums its rows' squares over its own eight columns for the v = 0 window
only, and since the column groups tile the template row, the v = 1 and v = 2
windows of a whole row differ from v = 0 by the frame columns t0 - 1, t0 at
the left end and t0 - 1 + n, t0 + n at the right end (values outside the
frame read as zero). Small random cases cover shifts past every edge."""
import numpy as np


def _sq(a, r, c):
    m, n = a.shape
    return int(a[r, c]) ** 2 if 0 <= r < m and 0 <= c < n else 0


def test_v0_window_plus_end_columns_equals_the_direct_sum():
    rng = np.random.default_rng(20150618)
    for _ in range(150):
        m = int(rng.integers(3, 14))
        n = 8 * int(rng.integers(1, 4))
        a = rng.integers(0, 65536, (m, n))
        s0 = int(rng.integers(-m - 1, m + 2))
        t0 = int(rng.integers(-n - 1, n + 2))
        i_b = int(rng.integers(0, m))
        i_e = min(m, i_b + int(rng.integers(1, 6)))
        L, first = i_e - i_b, i_b + s0 - 1
        for u in range(3):
            rows = range(first + u, first + u + L)  # frame rows of template rows i_b .. i_e-1
            v0 = sum(_sq(a, r, 8 * g + t0 - 1 + k) for g in range(n // 8) for r in rows for k in range(8))
            left = [(_sq(a, r, t0 - 1), _sq(a, r, t0)) for r in rows]
            right = [(_sq(a, r, t0 - 1 + n), _sq(a, r, t0 + n)) for r in rows]
            split = {0: v0,
                     1: v0 - sum(p for p, _ in left) + sum(p for p, _ in right),
                     2: v0 - sum(p + q for p, q in left) + sum(p + q for p, q in right)}
            for v in range(3):
                direct = sum(_sq(a, i + s0 - 1 + u, j + t0 - 1 + v) for i in range(i_b, i_e) for j in range(n))
                assert split[v] == direct, (m, n, s0, t0, i_b, i_e, u, v)
