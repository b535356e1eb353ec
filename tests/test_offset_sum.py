"""Host check of the offset accumulation the cluster QRP uses for A^T y over an FP32 A
(qrp_cluster.cu: off_fma, off_s1, off_s2), emulated exactly: every FP32 operation is
the exact rational result rounded to nearest-even FP32, in the kernel's order.

What the argument behind it claims, asserted here on random and cancelling inputs:
  - with s1 a power of two above 2 B (B >= every |partial sum| of a_i bh_i), the running
    sum hi stays in [s1/2, 3 s1/2] and hi - t is exact, so the FMA residual r is the
    rounding error of t to within 2^-24 |r|;
  - the residuals, summed around s2 (a power of two 4x above their largest possible
    sum), are summed exactly (Fast2Sum: r + (mid - t2) is the exact error of t2);
  - hi - s1 and mid - s2 are exact (Sterbenz);
  - the result is within k * 2^-48 * s1 of the exact sum of a_i (bh_i + bl_i)."""
import math
import random
from fractions import Fraction

import pytest


def rn32(x):
    """x (a Fraction) rounded to the nearest FP32 value, ties to even (normal and
    subnormal range; the inputs here stay far from overflow)."""
    if x == 0:
        return Fraction(0)
    sign = -1 if x < 0 else 1
    ax = -x if x < 0 else x
    e = ax.numerator.bit_length() - ax.denominator.bit_length()
    if Fraction(2) ** e > ax:
        e -= 1
    q = Fraction(2) ** (max(e, -126) - 23)  # the spacing of FP32 values around ax
    m = ax / q
    f = m.numerator // m.denominator
    rem = m - f
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and f % 2 == 1):
        f += 1
    return sign * f * q


def f32(v):
    return rn32(Fraction(v))


def fma(a, b, c):
    return rn32(a * b + c)


def add(a, b):
    return rn32(a + b)


def sub(a, b):
    return rn32(a - b)


def pow2_exp(x):
    """floor(log2 x) for x > 0 (the FP32 biased exponent minus 127 for normal x)."""
    e = x.numerator.bit_length() - x.denominator.bit_length()
    return e - 1 if Fraction(2) ** e > x else e


def off_sum(a, bh, bl):
    """The kernel's sequence for one column and one thread's rows."""
    k = len(a)
    # the bound: ||a|| ||bh|| with the kernel's 1 + 2^-8 margin (computed exactly here)
    na = math.sqrt(float(sum(x * x for x in a))) * (1 + 2.0 ** -8)
    ny = math.sqrt(float(sum(x * x for x in bh))) * (1 + 2.0 ** -8)
    nb = f32(na * ny)
    e1 = (pow2_exp(nb) + 127 + 2) if nb > 0 else 2  # biased exponent + 2, as off_s1
    e1 = min(max(e1, 1), 254)
    s1 = Fraction(2) ** (e1 - 127)
    lk = (k + 1).bit_length()  # 2^lk > rows per thread
    s2 = Fraction(2) ** (max(e1 - 22 + lk, 1) - 127)
    hi, mid, lo = s1, s2, Fraction(0)
    for ai, bhi, bli in zip(a, bh, bl):
        t = fma(ai, bhi, hi)
        d = sub(hi, t)
        assert d == hi - t, "hi - t must be exact"
        assert s1 / 2 <= t <= 3 * s1 / 2
        r = fma(ai, bhi, d)
        exact_r = ai * bhi + hi - t
        assert abs(r - exact_r) <= abs(exact_r) * Fraction(1, 2 ** 24)
        t2 = add(mid, r)
        e2 = sub(mid, t2)
        assert e2 == mid - t2, "mid - t2 must be exact"
        r2 = add(r, e2)
        assert r2 == r - (t2 - mid), "Fast2Sum: r2 is the exact error of t2"
        lo = fma(ai, bli, add(lo, r2))
        hi, mid = t, t2
    vh = sub(hi, s1)
    assert vh == hi - s1
    vm = sub(mid, s2)
    assert vm == mid - s2
    return vh + add(vm, lo), s1


def draw(rng, k, scale_a, scale_y, cancel=False):
    a, bh, bl, exact = [], [], [], Fraction(0)
    for i in range(k):
        av = f32(rng.gauss(0.0, 1.0) * scale_a)
        y = rng.gauss(0.0, 1.0) * scale_y
        if cancel and i % 2 == 1:  # undo the previous product to a few ulps: sums near zero
            av = -a[-1]
            y = float(bh[-1] + bl[-1]) * (1 + rng.uniform(-1e-7, 1e-7))
        h = f32(y)
        l_ = rn32(Fraction(y) - h)
        a.append(av)
        bh.append(h)
        bl.append(l_)
        exact += av * (h + l_)
    return a, bh, bl, exact


@pytest.mark.parametrize("k", [1, 7, 50, 200])
@pytest.mark.parametrize("cancel", [False, True])
def test_offset_sum_invariants_and_error(k, cancel):
    rng = random.Random(1000 * k + cancel)
    for trial in range(12 if k <= 50 else 4):
        scale_a = 2.0 ** rng.uniform(-20, 20)
        scale_y = 2.0 ** rng.uniform(-20, 20)
        a, bh, bl, exact = draw(rng, k, scale_a, scale_y, cancel)
        got, s1 = off_sum(a, bh, bl)
        bound = k * s1 / 2 ** 48
        assert abs(got - exact) <= bound, f"k={k} trial {trial}: error {float(abs(got - exact) / s1):.3e} s1"


def test_offset_sum_of_zeros_is_zero():
    got, _ = off_sum([Fraction(0)] * 5, [f32(0.5)] * 5, [Fraction(0)] * 5)
    assert got == 0
    got, _ = off_sum([f32(1.5)] * 3, [Fraction(0)] * 3, [Fraction(0)] * 3)
    assert got == 0


def test_rn32_matches_known_values():
    assert rn32(Fraction(1, 3)) == Fraction(11184811, 2 ** 25)  # 0x3eaaaaab
    assert rn32(Fraction(2 ** 24 + 1)) == 2 ** 24  # tie to even
    assert rn32(Fraction(2 ** 24 + 3)) == 2 ** 24 + 4
    assert rn32(Fraction(1, 2 ** 149)) == Fraction(1, 2 ** 149)  # smallest subnormal
