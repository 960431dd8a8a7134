"""The precision reading of the mixed path's residuals, pinned on the CPU.

The one-warp kernel forms the residual mat-vecs of its mixed-precision solve
in double-float on the FP32 pipe: each FP64 value is split into its FP32
rounding and the FP32 rounding of the remainder, each product is formed by an
exact FP32 product plus its FMA error and the two cross terms, and the sum is
carried by Knuth's two-sum in a high word while the errors gather in a low
word (two independent chains per row, joined at the end).  The claim is that
this keeps each row's error near 1e-14 of the sum of the terms' magnitudes
(FP64 gives about 1e-16), far below the refinement target of 1e-12 relative
to the right-hand side.  These tests restate the arithmetic in numpy float32,
operation by operation, and measure its error against exact rational sums.

Python floats are IEEE doubles and numpy float32 operations round to nearest,
so the restatement rounds where the kernel rounds.  The FMA steps are formed
in FP64 (a float32 product is exact there) and rounded to float32: exact for
the product's error term, and for the cross terms a double rounding that can
differ from a fused FMA in the last bit of a term far below the row's error.
"""
from fractions import Fraction

import numpy as np

f32 = np.float32


def split(x: float):
    h = f32(x)
    return h, f32(x - float(h))


def fma32(a, b, c):
    """float32 a * b + c, formed in FP64 and rounded to float32."""
    return f32(float(a) * float(b) + float(c))


def df_acc(ah, al, xh, xl, sh, sl):
    p = f32(ah * xh)
    e = fma32(ah, xh, -p)
    e = fma32(ah, xl, e)
    e = fma32(al, xh, e)
    t = f32(sh + p)
    bp = f32(t - sh)
    err = f32(f32(sh - f32(t - bp)) + f32(p - bp))
    return t, f32(sl + f32(err + e))


def df_join(h0, l0, h1, l1):
    t = f32(h0 + h1)
    bp = f32(t - h0)
    err = f32(f32(h0 - f32(t - bp)) + f32(h1 - bp))
    return float(t) + float(f32(f32(l0 + l1) + err))


def df_dot(a, x):
    """The kernel's row: two chains over even and odd terms, then joined."""
    h = [f32(0), f32(0)]
    l = [f32(0), f32(0)]
    for k, (ai, xi) in enumerate(zip(a, x)):
        ah, al = split(float(ai))
        xh, xl = split(float(xi))
        h[k & 1], l[k & 1] = df_acc(ah, al, xh, xl, h[k & 1], l[k & 1])
    return df_join(h[0], l[0], h[1], l[1])


def rel_errors(n, trials, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(trials):
        # magnitudes spread over six decades, as in a stage Hessian row times an iterate
        a = rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n))
        x = rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n))
        exact = sum(Fraction(float(ai)) * Fraction(float(xi)) for ai, xi in zip(a, x))
        scale = float(np.sum(np.abs(a * x)))
        out.append(abs(float(Fraction(df_dot(a, x)) - exact)) / scale)
    return np.array(out)


def test_split_carries_about_48_bits():
    rng = np.random.default_rng(1)
    for v in rng.standard_normal(200) * np.exp(rng.uniform(-20, 20, 200)):
        h, l = split(float(v))
        assert abs((float(h) + float(l)) - v) <= 2.0 ** -47 * abs(v)


def test_row_error_is_near_1e_minus_14_of_the_terms():
    # row lengths of the mass-spring stage (nu + nx = 23) and of a row with
    # its dynamics part (23 + 16 = 39 terms)
    for n in (23, 39):
        err = rel_errors(n, 150, seed=n)
        assert err.max() < 1e-13, err.max()
        assert np.median(err) < 1e-14, np.median(err)


def test_error_free_steps_are_exact():
    # two-sum and the FMA product error recover a + b and a * b exactly
    rng = np.random.default_rng(2)
    for _ in range(500):
        a, b = f32(rng.standard_normal() * 10.0 ** rng.integers(-5, 5)), f32(rng.standard_normal())
        t = f32(a + b)
        bp = f32(t - a)
        err = f32(f32(a - f32(t - bp)) + f32(b - bp))
        assert Fraction(float(t)) + Fraction(float(err)) == Fraction(float(a)) + Fraction(float(b))
        p = f32(a * b)
        e = fma32(a, b, -p)
        assert Fraction(float(p)) + Fraction(float(e)) == Fraction(float(a)) * Fraction(float(b))


def test_a_dropped_error_term_is_caught():
    # the same row without the cross terms (a plain FP32 product): the error
    # grows to FP32 size, which these bounds reject
    rng = np.random.default_rng(3)
    a = rng.standard_normal(39) * np.exp(rng.uniform(-3, 3, 39))
    x = rng.standard_normal(39) * np.exp(rng.uniform(-3, 3, 39))
    exact = sum(Fraction(float(ai)) * Fraction(float(xi)) for ai, xi in zip(a, x))
    s = 0.0
    for ai, xi in zip(a, x):
        s += float(f32(ai) * f32(xi))
    assert abs(float(Fraction(s) - exact)) / float(np.sum(np.abs(a * x))) > 1e-10
