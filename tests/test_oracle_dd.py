"""Pins for the double-double helpers (Sec. 2.2) against exact rational arithmetic."""
from fractions import Fraction as F

import numpy as np

from oracle import ddarith as dd


def _rand(g, n, spread=30):
    return g.standard_normal(n) * np.exp2(g.integers(-spread, spread, n))


def test_two_sum_exact():
    g = np.random.default_rng(1)
    a, b = _rand(g, 2000), _rand(g, 2000)
    x, y = dd.two_sum(a, b)
    for ai, bi, xi, yi in zip(a, b, x, y):
        assert F(ai) + F(bi) == F(xi) + F(yi)
        assert xi == ai + bi


def test_two_prod_exact():
    g = np.random.default_rng(2)
    a, b = _rand(g, 2000), _rand(g, 2000)
    p, e = dd.two_prod(a, b)
    for ai, bi, pi, ei in zip(a, b, p, e):
        assert F(ai) * F(bi) == F(pi) + F(ei)


def test_pair_add_matches_definition():
    # Sec. 2.2: [c_h, t] = TwoSum(a, b_h), c_l = fl(b_l + t); error only from the final add
    g = np.random.default_rng(3)
    a = g.standard_normal(500)
    bh = g.standard_normal(500)
    bl = bh * 2.0 ** -60 * g.standard_normal(500)
    ch, cl = dd.pair_add(a, bh, bl)
    for i in range(500):
        exact = F(a[i]) + F(bh[i]) + F(bl[i])
        err = abs(F(ch[i]) + F(cl[i]) - exact)
        assert err <= abs(exact) * F(2) ** -100 + F(2) ** -1074


def test_dd_matmul_against_fractions():
    g = np.random.default_rng(4)
    L = g.standard_normal((5, 7))
    Ll = L * 2.0 ** -55 * g.standard_normal((5, 7))
    R = g.standard_normal((7, 4))
    h, l = dd.dd_matmul(L, Ll, R, None)
    for i in range(5):
        for j in range(4):
            ex = sum(((F(L[i, k]) + F(Ll[i, k])) * F(R[k, j]) for k in range(7)), F(0))
            mag = sum((abs(F(L[i, k]) * F(R[k, j])) for k in range(7)), F(0))
            assert abs(F(h[i, j]) + F(l[i, j]) - ex) <= mag * F(2) ** -100


def test_dd_div():
    g = np.random.default_rng(5)
    a = g.standard_normal(200)
    b = 1.0 + 1e-3 * g.standard_normal(200)
    bl = b * 2.0 ** -60
    q = dd.dd_div_dd(a, np.zeros(200), b, bl)
    for i in range(200):
        ex = F(a[i]) / (F(b[i]) + F(bl[i]))
        assert abs(F(q[0][i]) + F(q[1][i]) - ex) <= abs(ex) * F(2) ** -100


def test_dd_sum_against_fractions():
    # the column sums of the residual step (x^T x, x^T v, r_ij) are double-double sums of
    # double-double terms; the chain of dd additions stays within about 2^-100 of the exact
    # sum, relative to the sum of the terms' magnitudes
    g = np.random.default_rng(6)
    h = g.standard_normal((64, 9))
    l = h * 2.0 ** -58 * g.standard_normal((64, 9))
    sh, sl = dd.dd_sum(h, l, axis=0)
    for j in range(9):
        ex = sum((F(h[k, j]) + F(l[k, j]) for k in range(64)), F(0))
        mag = sum((abs(F(h[k, j])) for k in range(64)), F(0))
        assert abs(F(sh[j]) + F(sl[j]) - ex) <= mag * F(2) ** -100


def test_dd_add_relative_bound_under_cancellation():
    # The accurate double-double sum (two TwoSums, a renormalisation, the low error term and a
    # second renormalisation) has relative error at most 3u^2 + 13u^3, u = 2^-53 (Joldes,
    # Muller and Popescu, ACM TOMS 2017), even when the high words cancel.  Exact cancellation
    # leaves the sum of the two low words, which a double-double holds exactly.
    g = np.random.default_rng(7)
    u = F(2) ** -53
    n = 400
    ah = g.standard_normal(n)
    al = ah * 2.0 ** -54 * g.uniform(-1, 1, n)
    bh = -ah * (1.0 + 2.0 ** -40 * g.standard_normal(n))
    bh[: n // 2] = -ah[: n // 2]                        # exact cancellation of the high words
    bl = bh * 2.0 ** -54 * g.uniform(-1, 1, n) * 2.0 ** -int(g.integers(0, 40))
    rh, rl = dd.dd_add(ah, al, bh, bl)
    for i in range(n):
        ex = F(ah[i]) + F(al[i]) + F(bh[i]) + F(bl[i])
        got = F(rh[i]) + F(rl[i])
        assert abs(got - ex) <= abs(ex) * (3 * u * u + 13 * u ** 3), i
        if i < n // 2:
            assert got == F(al[i]) + F(bl[i]), i
