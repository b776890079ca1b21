"""The double-single product used for the outer q = A p of the mixed-precision
solve, emulated step by step in FP32 on the CPU, against exact rational
arithmetic: a row of n terms stays within n * 2^-47 of sum |a x| of the exact
sum (the bound the GPU test's 2^-40 is derived from), and far inside the
2^-24 of a plain FP32 product.

Emulation: FP32 products and sums are numpy float32 operations (IEEE round to
nearest); the error of an FP32 product, e = a_hi x_hi - fl(a_hi x_hi), is
formed exactly from the float64 product of the two FP32 factors (48
significant bits) and is itself an FP32 number, which is what the kernel's
fma(a_hi, x_hi, -p) yields.
"""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32


def round_f32(q):
    """q (a Fraction) rounded to the nearest FP32 number, ties to even"""
    f = f32(float(q))
    cands = (f, np.nextafter(f, f32(np.inf)), np.nextafter(f, f32(-np.inf)))
    return min(cands, key=lambda c: (abs(Fraction(float(c)) - q),
                                     int(np.array(c, dtype=np.float32).view(np.uint32)) & 1))


def fma_f32(a, b, c):
    """fl32(a * b + c) with one rounding, for FP32 a, b, c"""
    return round_f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def split(v):
    hi = np.asarray(v, dtype=np.float64).astype(np.float32)
    lo = (np.asarray(v, dtype=np.float64) - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def ds_row(a, x):
    """s + t of the kernel's recurrence for one row (float64 result)"""
    ah, al = split(a)
    xh, xl = split(x)
    s, t = f32(0.0), f32(0.0)
    for c in range(len(a)):
        p = f32(ah[c] * xh[c])
        e = f32(np.float64(ah[c]) * np.float64(xh[c]) - np.float64(p))
        cross = fma_f32(ah[c], xl[c], f32(al[c] * xh[c]))
        s1 = f32(s + p)
        bp = f32(s1 - s)
        err = f32(f32(s - f32(s1 - bp)) + f32(p - bp))
        s = s1
        t = f32(t + f32(err + f32(e + cross)))
    return np.float64(s) + np.float64(t)


@pytest.mark.parametrize("n,seed,spread", [(10, 1, 0.0), (40, 2, 0.0), (140, 3, 3.0), (700, 4, 0.0),
                                           (700, 5, 6.0)])
def test_double_single_row_within_bound(n, seed, spread):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(n) * 10.0 ** rng.uniform(-spread, spread, n)
    x = rng.standard_normal(n)
    exact = sum(Fraction(float(ai)) * Fraction(float(xi)) for ai, xi in zip(a, x))
    absum = float(np.sum(np.abs(a * x)))
    got = ds_row(a, x)
    err = abs(Fraction(float(got)) - exact)
    assert float(err) <= n * 2.0 ** -47 * absum
    # a plain FP32 product of the same row is orders of magnitude worse
    p32 = f32(0.0)
    for ai, xi in zip(a.astype(np.float32), x.astype(np.float32)):
        p32 = f32(p32 + f32(ai * xi))
    assert float(abs(Fraction(float(p32)) - exact)) > 1e3 * float(err)


def test_split_is_exact_to_2_pow_48():
    rng = np.random.default_rng(7)
    v = rng.standard_normal(1000) * 10.0 ** rng.uniform(-5, 5, 1000)
    hi, lo = split(v)
    rel = np.abs(hi.astype(np.float64) + lo.astype(np.float64) - v) / np.abs(v)
    assert np.max(rel) <= 2.0 ** -48


def ds_dense_row(m, x, threads=256):
    """the dense bottom operator's row product in the FP32 cycle: m as its exact
    FP32 split, x exact in FP32, thread t runs the double-single recurrence over
    columns t, t + threads, ...; the threads' s + t pairs are added in FP64"""
    mh, ml = split(m)
    xf = np.asarray(x, dtype=np.float32)
    parts = []
    for t0 in range(threads):
        s, t = f32(0.0), f32(0.0)
        for c in range(t0, len(m), threads):
            p = f32(mh[c] * xf[c])
            e = f32(np.float64(mh[c]) * np.float64(xf[c]) - np.float64(p))
            cross = f32(ml[c] * xf[c])
            s1 = f32(s + p)
            bp = f32(s1 - s)
            err = f32(f32(s - f32(s1 - bp)) + f32(p - bp))
            s = s1
            t = f32(t + f32(err + f32(e + cross)))
        parts.append(np.float64(s) + np.float64(t))
    return float(np.sum(np.array(parts)))


@pytest.mark.parametrize("n,seed,spread", [(512, 6, 0.0), (2048, 7, 4.0)])
def test_double_single_dense_row_within_bound(n, seed, spread):
    """A row of the 2,048-dof bottom operator applied to an FP32 vector agrees
    with the exact FP64-operand product to within n * 2^-47 of sum |m x|."""
    rng = np.random.default_rng(seed)
    m = rng.standard_normal(n) * 10.0 ** rng.uniform(-spread, spread, n)
    x = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    exact = sum(Fraction(float(mi)) * Fraction(float(xi)) for mi, xi in zip(m, x))
    absum = float(np.sum(np.abs(m * x)))
    got = ds_dense_row(m, x)
    assert float(abs(Fraction(got) - exact)) <= n * 2.0 ** -47 * absum


def test_fma_emulation_rounds_once():
    """A case where rounding a*b + c first to float64 and then to FP32 differs
    from one rounding: the exact sum lies 2^-70 below the midpoint between
    two FP32 neighbours, so float64 lands on the midpoint and ties to even
    (up), while the single rounding goes down."""
    a = f32(2.0 ** -12 * (1 + 2.0 ** -23))
    b = f32(2.0 ** -12 * (1 - 2.0 ** -23))
    c = f32(1 + 2.0 ** -23)
    exact = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    mid = 1 + Fraction(1, 2 ** 23) + Fraction(1, 2 ** 24)
    assert mid - exact == Fraction(1, 2 ** 70)
    assert Fraction(float(fma_f32(a, b, c))) == 1 + Fraction(1, 2 ** 23)
    twice = f32(np.float64(a) * np.float64(b) + np.float64(c))
    assert Fraction(float(twice)) == 1 + Fraction(1, 2 ** 22)
