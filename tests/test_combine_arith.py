"""The FP32 combine's arithmetic, emulated on the host with IEEE float32
operations in the order the kernels issue them (no multiply feeds an add, so
no fused multiply-add can change a rounding):

* energy_pair: an exact energy e < 2^53 as three exact FP32 limbs and an
  error-free sum; hi + lo must equal e to within 2^-24 |lo| (exactly for
  e < 2^24);
* combine_f32: f = (Sa + Sb - 2h) * (unit / Area) from the two pairs, TwoSum
  on the high parts; relative to the exact value of the same expression
  (the given h and unit / Area taken as exact) the error must stay within a
  few units of FP32 rounding even when Sa + Sb and 2h cancel to 1e-7 of
  their size, the case where an FP32 sum of the energies would be useless;
* f32_to_f64: the bit move equals the conversion for normal floats.
"""
from fractions import Fraction

import numpy as np
import pytest

F = np.float32
U = 2.0 ** -24


def small_u32_to_float(x):
    return (np.array([0x4B000000 | int(x)], np.uint32).view(np.float32)[0] - F(8388608.0)).astype(F)


def energy_pair(e):
    H, L = e >> 32, e & 0xFFFFFFFF
    e2 = F(small_u32_to_float(H) * F(4294967296.0))
    e1 = F(small_u32_to_float(L >> 16) * F(65536.0))
    e0 = small_u32_to_float(L & 0xFFFF)
    hi = F(e2 + e1)
    bb = F(hi - e2)
    r = F(F(e2 - F(hi - bb)) + F(e1 - bb))
    return hi, F(r + e0)


def combine_f32(sa, sb, h, ia):
    s = F(sa[0] + sb[0])
    bb = F(s - sa[0])
    err = F(F(sa[0] - F(s - bb)) + F(sb[0] - bb))
    num = F(F(s - F(F(2.0) * h)) + F(err + F(sa[1] + sb[1])))
    return F(num * ia)


def fr(x):
    return Fraction(float(x))


def test_energy_pair_exact_limbs():
    rng = np.random.default_rng(7)
    cases = [0, 1, 2 ** 24 - 1, 2 ** 24, 2 ** 24 + 1, 2 ** 32 - 1, 2 ** 32, 2 ** 40 + 12345, 2 ** 53 - 1]
    cases += [int(x) for x in rng.integers(0, 2 ** 53, 2000, dtype=np.int64)]
    cases += [int(x) for x in rng.integers(0, 2 ** 30, 500, dtype=np.int64)]
    for e in cases:
        hi, lo = energy_pair(e)
        err = abs(fr(hi) + fr(lo) - e)
        assert err <= Fraction(abs(float(lo))) * Fraction(1, 2 ** 24), (e, hi, lo)
        if e < 2 ** 24:
            assert err == 0
        assert abs(float(lo)) <= abs(float(hi)) * 2.0 ** -24 + 2 ** 16 + 1  # lo: the bottom limb and a rounding


@pytest.mark.parametrize("rel_gap", [1e-1, 1e-4, 1e-7, 0.0])
def test_combine_error_relative_to_f_under_cancellation(rel_gap):
    # Sa + Sb and 2h agree to rel_gap: f = (Sa + Sb - 2h) / Area is rel_gap of
    # the energies' size. The combine's own error must be a few u of f (plus
    # nothing when f = 0 exactly).
    rng = np.random.default_rng(int(rel_gap * 1e9) + 3)
    worst = 0.0
    for _ in range(3000):
        lo_e = int(rng.choice([10, 20, 30]))
        sa = int(rng.integers(2 ** lo_e, 2 ** 46))
        sb = int(rng.integers(2 ** lo_e, 2 ** int(rng.choice([lo_e + 4, 46]))))
        h = F((sa + sb) * (1.0 - rel_gap * rng.uniform(0.5, 1.0)) / 2.0)
        area = int(rng.integers(1000, 70000))
        ia = F(1.0 / area)
        exact = (sa + sb - 2 * fr(h)) * fr(ia)
        got = combine_f32(energy_pair(sa), energy_pair(sb), h, ia)
        if exact == 0:
            assert float(got) == 0.0 or abs(float(got)) <= 2 * U * (sa + sb) * float(ia) * 2 ** -20
            continue
        rel = abs(fr(got) - exact) / abs(exact)
        worst = max(worst, float(rel))
    assert worst <= 3 * U, worst


def test_f32_to_f64_bit_move_equals_conversion():
    rng = np.random.default_rng(11)
    xs = np.concatenate([rng.standard_normal(1000).astype(F) * F(1e3), np.array([1.0, -2.5, 3e38, 1.2e-38], F)])
    for x in xs:
        u = int(np.array([x], F).view(np.uint32)[0])
        ex = (u >> 23) & 0xFF
        if ex in (0, 0xFF):
            continue
        bits = ((u & 0x80000000) << 32) | ((ex + 896) << 52) | ((u & 0x7FFFFF) << 29)
        assert np.array([bits], np.uint64).view(np.float64)[0] == np.float64(x)
