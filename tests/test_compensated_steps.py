"""The compensated float32 steps behind the float64 refinement (Q37), written
out in exact rational arithmetic with float32 rounding to nearest, on random
operands: the packed form used by the kernels (the product's negation q = -p
formed as ah * (-bh), TwoSum(s, p) written as (s - q, (s - (sn - bp)) -
(q + bp))) gives the same bits as the scalar form (Knuth's TwoSum of s and
p), and one compensated step adds (ah + al)(bh + bl) to the float pair
(s, c) with an error of a few 2^-47 of |s| + |ab|.

These check the algebra of the steps, not the CUDA kernels: the kernels'
results are compared with the oracle in the -m gpu tests."""
from fractions import Fraction

import numpy as np

F32 = np.float32


def r32(x: Fraction) -> np.float32:
    """x rounded to the nearest float32 (ties to even)."""
    c = F32(float(x))
    cands = [np.nextafter(c, F32(-np.inf)), c, np.nextafter(c, F32(np.inf))]

    def key(y):
        bits = int(np.frombuffer(np.float32(y).tobytes(), np.uint32)[0])
        return (abs(Fraction(float(y)) - x), bits & 1)

    return F32(min(cands, key=key))


def add(a, b):
    return r32(Fraction(float(a)) + Fraction(float(b)))


def sub(a, b):
    return r32(Fraction(float(a)) - Fraction(float(b)))


def mul(a, b):
    return r32(Fraction(float(a)) * Fraction(float(b)))


def fma(a, b, c):
    return r32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def mac_scalar(ah, al, bh, bl, s, c):
    p = mul(ah, bh)
    e = fma(ah, bh, -p)
    x = fma(ah, bl, mul(al, bh))
    sn = add(s, p)
    bp = sub(sn, s)
    t = add(sub(s, sub(sn, bp)), sub(p, bp))
    return sn, add(c, add(t, add(e, x)))


def mac_packed(ah, al, bh, bl, s, c):
    q = mul(ah, -bh)
    e = fma(ah, bh, q)
    x = fma(ah, bl, mul(al, bh))
    sn = sub(s, q)
    bp = sub(sn, s)
    t = sub(sub(s, sub(sn, bp)), add(q, bp))
    return sn, add(c, add(t, add(e, x)))


def operands(rng):
    """Float pairs as the splits make them: |al| <= 2^-24 |ah|, |bl| <=
    2^-24 |bh|, |c| <= 2^-24 |s|, magnitudes over six decades."""
    v = rng.standard_normal(3) * 10.0 ** rng.integers(-3, 3, 3)
    u = rng.uniform(-1.0, 1.0, 3) * 2.0 ** -24
    ah, bh, s = F32(v[0]), F32(v[1]), F32(v[2])
    al, bl, c = F32(float(ah) * u[0]), F32(float(bh) * u[1]), F32(float(s) * u[2])
    return ah, al, bh, bl, s, c


def test_packed_step_gives_the_scalar_bits():
    rng = np.random.default_rng(1)
    for _ in range(3000):
        args = operands(rng)
        a = mac_scalar(*args)
        b = mac_packed(*args)
        assert a[0] == b[0] and a[1] == b[1], args


def test_step_is_compensated():
    """(s', c') = step(s, c) satisfies s' + c' = s + c + (ah + al)(bh + bl)
    up to a few 2^-47 of |s| + |a b| (the neglected al bl and the roundings
    of the error terms)."""
    rng = np.random.default_rng(2)
    for _ in range(3000):
        ah, al, bh, bl, s, c = operands(rng)
        sn, cn = mac_packed(ah, al, bh, bl, s, c)
        exact = (Fraction(float(s)) + Fraction(float(c))
                 + (Fraction(float(ah)) + Fraction(float(al))) * (Fraction(float(bh)) + Fraction(float(bl))))
        got = Fraction(float(sn)) + Fraction(float(cn))
        scale = abs(float(s)) + abs(float(ah) * float(bh))
        assert abs(float(got - exact)) <= 8 * 2.0 ** -47 * scale + 1e-300, (ah, al, bh, bl, s, c)


def test_a_plain_float32_sum_is_not_enough():
    """The same sum taken as one float32 addition loses the low word: the
    compensation is what the steps are for."""
    rng = np.random.default_rng(3)
    worse = 0
    for _ in range(500):
        ah, al, bh, bl, s, c = operands(rng)
        exact = (Fraction(float(s)) + Fraction(float(c))
                 + (Fraction(float(ah)) + Fraction(float(al))) * (Fraction(float(bh)) + Fraction(float(bl))))
        plain = Fraction(float(add(s, mul(ah, bh))))
        sn, cn = mac_packed(ah, al, bh, bl, s, c)
        comp = Fraction(float(sn)) + Fraction(float(cn))
        worse += abs(plain - exact) > abs(comp - exact)
    assert worse > 450
