"""Pins for the Ozaki splitting and slice-product oracle (Sec. 2.3)."""
import math
from fractions import Fraction as F

import numpy as np
import pytest

from oracle import ozaki as oz
from paper_2602_19090_gb300 import synth

U = F(1, 2 ** 53)


def ufp(x):
    return F(2) ** math.floor(math.log2(abs(x))) if x != 0 else F(0)


def test_ceil_log2_exact():
    g = np.random.default_rng(11)
    m = np.abs(g.standard_normal(3000)) * np.exp2(g.integers(-300, 300, 3000))
    m[:50] = np.exp2(np.arange(-25, 25))          # exact powers of two
    e = oz.ceil_log2(m)
    for mi, ei in zip(m, e):
        assert F(2) ** (int(ei) - 1) < F(mi) <= F(2) ** int(ei)
    assert oz.ceil_log2(np.array([0.0]))[0] == oz.EZERO


@pytest.mark.parametrize("phi", [0.5, 2.0, 4.0])
def test_slices_round_trip_digits_and_residual_bound(phi):
    M = synth.gemm_operand(9, 23, phi, 7)
    M[3, :] = 0.0                                  # zero row: sigma = 0 (eq. sigma)
    k = 6
    d, e, res = oz.slice_rows(M, k)
    assert np.all(np.abs(d) <= 128)                  # 8-bit digits: |d| <= 2^7
    assert np.all(d[:, 3, :] == 0)
    for i in range(M.shape[0]):
        for j in range(M.shape[1]):
            acc = F(0)
            for r in range(1, k + 1):
                if e[i] != oz.EZERO:
                    acc += d[r - 1, i, j] * F(2) ** int(e[i] + 1 - 8 * r)
            assert acc + F(res[i, j]) == F(M[i, j])              # exact split
            if e[i] != oz.EZERO:
                assert abs(F(res[i, j])) <= F(2) ** int(e[i] - 8 * k)   # |res_k| <= w_k / 2


def test_digit_rule_is_the_sigma_trick():
    # eq. a: a^(r) = fl((sigma + a_res) - sigma) with ulp(sigma) = w_r gives the same slice
    M = synth.gemm_operand(16, 40, 2.0, 8)
    d, e, _ = oz.slice_rows(M, 7)
    res = M.copy()
    for r in range(1, 8):
        w = np.ldexp(1.0, e + 1 - 8 * r)[:, None]
        sl = oz.sigma_trick_slice(res, e, r)
        assert np.array_equal(d[r - 1] * w, sl)
        res = res - sl


def test_ties_go_to_even_digit():
    # e = 0 (max 1.0): w_1 = 2^-7; 1.0 is the largest digit, 128; 2.5 w_1 -> digit 2,
    # 3.5 w_1 -> 4
    x = np.array([[1.0, 2.5 * 2.0 ** -7, 3.5 * 2.0 ** -7, -2.5 * 2.0 ** -7]])
    d, e, _ = oz.slice_rows(x, 1)
    assert e[0] == 0
    assert list(d[0, 0]) == [128, 2, 4, -2]


@pytest.mark.parametrize("beta", [3, 10, 17, 30, 47])
def test_tau_truncation(beta):
    X = synth.gemm_operand(30, 12, 1.0, 9)
    X1, f = oz.tau_truncate_cols(X, beta)
    for j in range(X.shape[1]):
        tau = F(3, 4) * F(2) ** int(f[j] + beta)
        grid = F(2) ** int(f[j] + beta - 53)          # ulp(tau)
        for i in range(X.shape[0]):
            x1 = F(X1[i, j])
            assert (x1 / grid).denominator == 1
            assert abs(F(X[i, j]) - x1) <= U * ufp(tau)   # eq. minamihata
            q = F(X[i, j]) / grid                          # round to nearest, ties to even
            fl = math.floor(q)
            rnd = fl + (1 if (q - fl > F(1, 2) or (q - fl == F(1, 2) and fl % 2)) else 0)
            assert x1 == rnd * grid


def test_slice_products_fp64_route_is_exact_at_the_extremes():
    # all digits +-128 with K = 2048: partial sums reach K * 2^14 = 2^25; and a random sign
    # pattern checked against Python integers term by term on a few entries
    K = 2048
    dL = np.full((2, 3, K), 128, dtype=np.int64)
    dR = np.full((2, K, 4), 128, dtype=np.int64)
    dR[1] = -128
    S = oz.slice_products(dL, dR, oz.pair_set(2, 2, 4))
    assert int(S[2][0, 0]) == K * 16384
    assert int(S[3][0, 0]) == 0          # (1,2) gives -K 2^14, (2,1) gives +K 2^14
    assert int(S[4][0, 0]) == -K * 16384
    g = np.random.default_rng(13)
    dL = g.integers(-128, 129, (2, 3, 5000))
    dR = g.integers(-128, 129, (2, 5000, 3))
    S = oz.slice_products(dL, dR, oz.pair_set(2, 2, 4))
    for i in range(3):
        for j in range(3):
            ref = sum(int(a) * int(b) for a, b in zip(dL[0, i], dR[1, :, j])) + \
                  sum(int(a) * int(b) for a, b in zip(dL[1, i], dR[0, :, j]))
            assert int(S[3][i, j]) == ref


def test_slice_products_brute_force():
    g = np.random.default_rng(12)
    dL = g.integers(-128, 129, (3, 4, 6))
    dR = g.integers(-128, 129, (3, 6, 5))
    pairs = oz.pair_set(3, 3, 4)
    S = oz.slice_products(dL, dR, pairs)
    assert set(S) == {2, 3, 4}
    for t, St in S.items():
        for i in range(4):
            for j in range(5):
                ref = 0
                for (r, s) in pairs:
                    if r + s == t:
                        ref += sum(int(dL[r - 1, i, k]) * int(dR[s - 1, k, j]) for k in range(6))
                assert St[i, j] == ref


def _exact_product(A, B):
    m, K = A.shape
    n = B.shape[1]
    return [[sum((F(A[i, k]) * F(B[k, j]) for k in range(K)), F(0)) for j in range(n)] for i in range(m)]


def test_ozaki_gemm_enough_slices_is_correctly_rounded():
    A = synth.gemm_operand(6, 9, 0.5, 21)
    B = synth.gemm_operand(9, 5, 0.5, 22)
    # exponent spread is small; 12 planes (96 bits) capture both operands exactly
    _, eA, resA = oz.slice_rows(A, 12)
    _, eB, resB = oz.slice_cols(B, 12)
    assert np.all(resA == 0) and np.all(resB == 0)
    C, out = oz.ozaki_gemm(A, B, 12, "full", exact=True)
    ex = _exact_product(A, B)
    for i in range(6):
        for j in range(5):
            assert C[i, j] == float(ex[i][j])           # RN of the exact product
            assert F(out["hi"][i, j]) + F(out["lo"][i, j]) - ex[i][j] <= abs(ex[i][j]) * F(2) ** -104


def test_full_pair_set_is_exact_for_integer_operands():
    # Sec. 2.3: with every operand held exactly by its k planes, the product over all k^2
    # slice pairs is the exact product.  Integers below 2^23 need three 8-bit planes, and the
    # last pair (3, 3) carries the units digits, so the exact integer product tells whether
    # every pair was taken.
    g = np.random.default_rng(23)
    A = g.integers(-(1 << 23) + 1, 1 << 23, size=(6, 9)).astype(np.float64)
    B = g.integers(-(1 << 23) + 1, 1 << 23, size=(9, 5)).astype(np.float64)
    assert np.all(oz.slice_rows(A, 3)[2] == 0) and np.all(oz.slice_cols(B, 3)[2] == 0)
    C, out = oz.ozaki_gemm(A, B, 3, "full")
    assert len(out["pairs"]) == 9
    for i in range(6):
        for j in range(5):
            ex = sum(int(A[i, q]) * int(B[q, j]) for q in range(9))
            assert F(out["hi"][i, j]) + F(out["lo"][i, j]) == ex
            assert C[i, j] == float(ex)


@pytest.mark.parametrize("k", [2, 3, 4, 6])
def test_triangular_truncation_bound(k):
    A = synth.gemm_operand(7, 11, 2.0, 31)
    B = synth.gemm_operand(11, 6, 2.0, 32)
    C, out = oz.ozaki_gemm(A, B, k, "triangular", exact=True)
    assert len(out["pairs"]) == k * (k + 1) // 2
    ex = _exact_product(A, B)
    eA, eB = out["eL"], out["eR"]
    K = A.shape[1]
    for i in range(7):
        for j in range(6):
            # dropped pairs (r + s >= k + 2: |a_r b_s| <= 2^(eA + eB + 16 - 8(r + s)), at most k
            # per anti-diagonal, decaying by 2^-8) and the two residual terms (each below
            # 2^(eA + eB - 8k) per product term): (1.004 k + 2.01) K 2^(eA + eB - 8k)
            bound = (k + 3) * K * F(2) ** int(eA[i] + eB[j] - 8 * k)
            assert abs(F(out["hi"][i, j]) + F(out["lo"][i, j]) - ex[i][j]) <= bound


def test_recombine_dd_matches_exact():
    A = synth.gemm_operand(20, 30, 4.0, 41)
    B = synth.gemm_operand(30, 10, 4.0, 42)
    _, o1 = oz.ozaki_gemm(A, B, 10, "full", exact=True)
    _, o2 = oz.ozaki_gemm(A, B, 10, "full", exact=False)
    for t in o1["S"]:
        assert np.array_equal(o1["S"][t], o2["S"][t])
    mag = np.abs(A) @ np.abs(B)
    diff = np.abs((o1["hi"] - o2["hi"]) + (o1["lo"] - o2["lo"]))
    assert np.all(diff <= mag * 2.0 ** -100)


def _ufp(x):
    return F(2) ** (math.frexp(abs(float(x)))[1] - 1)


@pytest.mark.parametrize("phi", [0.5, 4.0])
def test_adaptive_slices_split_exactly_and_obey_eq_minamihata(phi):
    # the paper's own splitting (eq. sigma with a rescan before every slice, eq. a): the
    # slices and the residual add up to M exactly, and after slice r the residual is at most
    # u * ufp(sigma_i^(r)) (eq. minamihata); a zero row gets sigma = 0 and zero slices
    M = synth.gemm_operand(7, 19, phi, 50)
    M[2, :] = 0.0
    k, alpha = 3, 30
    sl, sig, res = oz.slice_rows_adaptive(M, k, alpha)
    assert np.all(sl[:, 2, :] == 0) and np.all(sig[:, 2] == 0)
    for i in range(M.shape[0]):
        for j in range(M.shape[1]):
            rem = F(M[i, j])
            for r in range(k):
                rem -= F(sl[r, i, j])
                if sig[r, i] != 0:
                    assert abs(rem) <= U * _ufp(sig[r, i])
            assert rem == F(res[i, j])


def test_adaptive_slice_products_are_exact_under_eq_alp_beta():
    # alpha + beta >= -log2 u + log2 n makes every slice product exact in FP64
    n = 16
    A = synth.gemm_operand(5, n, 2.0, 51)
    X = synth.gemm_operand(n, 4, 2.0, 52)
    alpha = 30
    beta = 53 + 4 - alpha
    sa, _, _ = oz.slice_rows_adaptive(A, 3, alpha)
    sx, _, _ = oz.slice_rows_adaptive(X.T, 3, beta)
    for r in range(3):
        for s in range(3):
            P = sa[r] @ sx[s].T
            for i in range(5):
                for j in range(4):
                    exact = sum((F(sa[r, i, q]) * F(sx[s, j, q]) for q in range(n)), F(0))
                    assert F(P[i, j]) == exact


@pytest.mark.parametrize("phi", [0.5, 2.0, 4.0])
def test_adaptive_slicing_needs_no_more_slices_than_the_fixed_grid(phi):
    # alpha = 46 gives slices of at most 2^7 units of ulp(sigma), the width of the fixed
    # 8-bit digit grid: the rescan starts every slice at the residual's leading bit, so it
    # represents each row exactly with at most as many slices as the fixed grid's planes
    M = synth.gemm_operand(24, 20, phi, 53)
    for i in range(M.shape[0]):
        row = M[i:i + 1]
        kf = next((k for k in range(1, 20) if np.all(oz.slice_rows(row, k)[2] == 0)), None)
        ka = next((k for k in range(1, 20) if np.all(oz.slice_rows_adaptive(row, k, 46)[2] == 0)), None)
        assert kf is not None, i
        assert ka is not None and ka <= kf, (i, ka, kf)      # None: never exact within 19 slices


def test_product_counts_printed_in_the_paper():
    # tests/golden/paper_product_counts.json: the counts Sec. 2.3 and Sec. 4.1 print
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_product_counts.json")))
    tri = g["triangular_products"]
    for k, p, a in zip(tri["k"], tri["products"], tri["additions"]):
        pairs = oz.pair_set(k, k, k + 1)
        assert len(pairs) == p
        # the exact sums add every product but the first of its anti-diagonal into it, then
        # the anti-diagonals into each other: (pairs - diagonals) + (diagonals - 1) additions
        diagonals = len({r + s for r, s in pairs})
        assert (len(pairs) - diagonals) + (diagonals - 1) == a
    prev = g["previous_study"]
    assert len(oz.pair_set(prev["n_A"], prev["n_X"], prev["n_A"] + 1)) == prev["products"]
    pro = g["proposed"]
    n_eq = pro["equal_cost_n_A"]
    # n_X = 1: the accurate A X^(1) takes n_A products (one per slice of A)
    assert len(oz.pair_set(n_eq, pro["n_X"], n_eq + 1)) == n_eq
    # both forms add the same two products per iteration, so the costs meet where the A X
    # products do: n_A = the previous study's six
    assert n_eq == prev["products"]
