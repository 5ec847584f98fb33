"""Ozaki-scheme error-free splitting and exact slice products (Sec. 2.3).

ORACLE: test infrastructure only.

Reading of eq. sigma and eq. a used throughout (the "digit grid"):
for a vector with maximum magnitude v > 0 let e = ceil(log2 v) (so v <= 2^e);
slice r of an entry is taken on the grid w_r = 2^(e + 1 - 8r) (DIGIT_BITS = 8
bits per slice).  This is the paper's sigma-trick a^(r) = fl((sigma + a_res) - sigma)
with a fixed sigma_r = 0.75 * 2^(e + 54 - 8r) (ulp(sigma_r) = w_r) instead of a
rescan of the residual's maximum, so every slice is an integer digit d with
|d| <= 128 times w_r, exact in bfloat16 (whose 8-bit significand holds every
integer up to 256).  Residuals obey |res_r| <= w_r / 2 = 2^(e - 8r), the analogue
of eq. minamihata.
A zero vector gets exponent EZERO and all-zero digits (sigma = 0 in eq. sigma).

A product C = L R with L sliced by rows (exponents eL_i) and R by columns (eR_j)
is  C_ij = sum_{(r,s)} 2^(eL_i + eR_j + 2 - 8(r+s)) * sum_k dL_r[i,k] dR_s[k,j],
the inner sums being exact integers (eq. after alp_beta: every slice product is
exact).  The pair set keeps r + s <= T (T = kL + kR: all pairs; T = k + 1: the
triangular k(k+1)/2 form cited after eq. alp_beta).
"""
from __future__ import annotations

import math

import numpy as np

from . import ddarith as dd

EZERO = -(1 << 30)   # exponent of an all-zero vector
DIGIT_BITS = 8       # bits per digit plane (|digit| <= 2^(DIGIT_BITS - 1) = 128)
DIGIT_MAX = 1 << (DIGIT_BITS - 1)
MAX_PLANES = 16      # planes per operand (128 bits)


def ceil_log2(m):
    """Exact ceil(log2 m) for m > 0 (array); EZERO where m == 0.

    m = fr * 2^ex with fr in [0.5, 1): ceil(log2 m) = ex, or ex - 1 if fr == 0.5.
    """
    m = np.asarray(m, dtype=np.float64)
    fr, ex = np.frexp(m)
    e = np.where(fr == 0.5, ex - 1, ex).astype(np.int64)
    return np.where(m == 0.0, EZERO, e)


def row_exponents(M):
    """e_i = ceil(log2 max_j |m_ij|) (eq. sigma's exponent)."""
    return ceil_log2(np.max(np.abs(M), axis=1)) if M.shape[1] else np.full(M.shape[0], EZERO)


def col_exponents(M):
    """f_j = ceil(log2 max_i |m_ij|) (eq. tau's exponent)."""
    return row_exponents(M.T)


def plane_weight(e, r):
    """w_r = 2^(e + 1 - DIGIT_BITS r); 0 for a zero vector."""
    e = np.asarray(e, dtype=np.int64)
    w = np.ldexp(1.0, np.where(e == EZERO, 0, e + 1 - DIGIT_BITS * r))
    return np.where(e == EZERO, 0.0, w)


def slice_rows(M, k, e=None):
    """Digit planes of M by rows: M = sum_{r<=k} d_r * w_r(e_i) + res.

    Returns (digits int64 [k, m, K], e int64 [m], residual FP64 [m, K]).
    d_r = rint(res / w_r) (round half to even), res <- res - d_r w_r; both steps
    are exact in FP64 because w_r is a power of two.
    """
    M = np.asarray(M, dtype=np.float64)
    if e is None:
        e = row_exponents(M)
    res = M.copy()
    digits = np.zeros((k,) + M.shape, dtype=np.int64)
    zero = (e == EZERO)
    for r in range(1, k + 1):
        w = plane_weight(e, r)[:, None]
        ws = np.where(w == 0.0, 1.0, w)
        d = np.rint(res / ws)
        d[zero, :] = 0.0
        res = res - d * w
        digits[r - 1] = d.astype(np.int64)
    return digits, e, res


def slice_cols(M, k, f=None):
    """Digit planes of M by columns. Returns (digits [k, K, n], f [n], residual)."""
    d, f, res = slice_rows(np.asarray(M).T, k, f)
    return np.transpose(d, (0, 2, 1)), f, res.T


def sigma_trick_slice(res, e, r):
    """Eq. a with sigma_r = 0.75 * 2^(e + 54 - DIGIT_BITS r): fl((sigma + res) - sigma), per row."""
    e = np.asarray(e, dtype=np.int64)
    sig = np.where(e == EZERO, 0.0, 0.75 * np.ldexp(1.0, np.where(e == EZERO, 0, e + 54 - DIGIT_BITS * r)))
    sig = sig[:, None]
    return (sig + res) - sig


def slice_rows_adaptive(M, k, alpha):
    """The paper's own splitting (eq. sigma and eq. a, Sec. 2.3), row by row, k slices.

    Before every slice the residual's row maximum v_i^(r) is scanned again and
    sigma_i^(r) = 0.75 * 2^ceil(log2 v_i^(r)) * 2^alpha (0 for a zero row); the slice is
    a^(r) = fl((sigma + res) - sigma) and the residual res <- fl(res - a^(r)).  Each slice
    keeps the bits of the residual from its leading one down to ulp(sigma), i.e. about
    53 - alpha bits, so its width follows the data instead of a fixed grid.

    Returns (slices FP64 [k, m, K], sigmas [k, m], residual [m, K]).
    (The CUDA path keeps the fixed grid of ``slice_rows``: a per-slice rescan gives every
    row its own slice exponents, which would break the anti-diagonal grouping of the exact
    integer sums.  This function is the reference for comparing the two.)
    """
    M = np.asarray(M, dtype=np.float64)
    res = M.copy()
    slices = np.zeros((k,) + M.shape)
    sigmas = np.zeros((k, M.shape[0]))
    for r in range(k):
        v = np.max(np.abs(res), axis=1) if M.shape[1] else np.zeros(M.shape[0])
        e = ceil_log2(v)
        sig = np.where(e == EZERO, 0.0, 0.75 * np.ldexp(1.0, np.where(e == EZERO, 0, e + alpha)))
        sl = (sig[:, None] + res) - sig[:, None]
        res = res - sl
        slices[r] = sl
        sigmas[r] = sig
    return slices, sigmas, res


def tau_truncate_cols(X, beta, f=None):
    """Eq. tau / eq. x with s = 1: X^(1)_ij = fl((tau_j + x_ij) - tau_j),

    tau_j = 0.75 * 2^(f_j) * 2^beta (0 for a zero column).
    Returns (X1, f).
    """
    X = np.asarray(X, dtype=np.float64)
    if f is None:
        f = col_exponents(X)
    tau = np.where(f == EZERO, 0.0, 0.75 * np.ldexp(1.0, np.where(f == EZERO, 0, f + beta)))
    tau = tau[None, :]
    return (tau + X) - tau, f


def pair_set(kL, kR, T):
    """All (r, s) with 1 <= r <= kL, 1 <= s <= kR, r + s <= T."""
    return [(r, s) for r in range(1, kL + 1) for s in range(1, kR + 1) if r + s <= T]


def slice_products(dL, dR, pairs):
    """S_t = sum over pairs with r + s = t of dL_r @ dR_s, exact int64 matrices.

    Every entry of dL_r @ dR_s is a sum of K integer terms of magnitude <= 128 * 128 = 2^14,
    so all its partial sums are integers of magnitude <= K * 2^14.  While that bound is
    below 2^53 an FP64 matrix product is exact whatever its summation order, and the
    library routine evaluates it; otherwise the products are taken in int64.
    """
    S = {}
    K = dL.shape[-1]
    exact_f64 = K * DIGIT_MAX * DIGIT_MAX < 2 ** 53
    if exact_f64:
        fL = dL.astype(np.float64)
        fR = dR.astype(np.float64)
    for (r, s) in pairs:
        if exact_f64:
            P = (fL[r - 1] @ fR[s - 1]).astype(np.int64)
        else:
            P = dL[r - 1] @ dR[s - 1]
        t = r + s
        S[t] = S[t] + P if t in S else P
    return S


def _scale_exponents(eL, eR, t):
    eL = np.asarray(eL, dtype=np.int64)[:, None]
    eR = np.asarray(eR, dtype=np.int64)[None, :]
    zero = (eL == EZERO) | (eR == EZERO)
    ex = np.where(zero, 0, eL + eR + 2 - DIGIT_BITS * t)
    return ex, zero


def recombine_dd(S, eL, eR, shape):
    """sum_t S_t * 2^(eL_i + eR_j + 2 - DIGIT_BITS t) as a double-double.

    Terms are added from the least significant t upwards with TwoSum; each term
    is exact in FP64 (|S_t| < 2^53 is asserted).
    """
    hi = np.zeros(shape)
    lo = np.zeros(shape)
    for t in sorted(S.keys(), reverse=True):
        St = S[t]
        assert np.all(np.abs(St) < (1 << 53))
        ex, zero = _scale_exponents(eL, eR, t)
        term = np.where(zero, 0.0, np.ldexp(St.astype(np.float64), ex))
        hi, lo = dd.dd_add_d(hi, lo, term)
    return hi, lo


def recombine_exact(S, eL, eR, shape):
    """Same sum, rounded exactly: hi = RN(sum), lo = RN(sum - hi) (math.fsum per entry).

    Pure-Python loop: small inputs only.
    """
    ts = sorted(S.keys())
    exps = {}
    for t in ts:
        ex, zero = _scale_exponents(eL, eR, t)
        exps[t] = (np.broadcast_to(ex, shape), np.broadcast_to(zero, shape))
    hi = np.zeros(shape)
    lo = np.zeros(shape)
    for i in range(shape[0]):
        for j in range(shape[1]):
            terms = [math.ldexp(float(S[t][i, j]), int(exps[t][0][i, j]))
                     for t in ts if not exps[t][1][i, j]]
            h = math.fsum(terms)
            hi[i, j] = h
            lo[i, j] = math.fsum(terms + [-h])
    return hi, lo


def ozaki_product(L, R, kL, kR, T, eL=None, eR=None, exact=False):
    """Accurate product C ~= L R from kL row planes of L, kR column planes of R,
    pairs r + s <= T.  Returns dict(hi, lo, S, dL, dR, eL, eR, pairs).
    """
    dL, eL, _ = slice_rows(L, kL, eL)
    dR, eR, _ = slice_cols(R, kR, eR)
    pairs = pair_set(kL, kR, T)
    S = slice_products(dL, dR, pairs)
    shape = (np.shape(L)[0], np.shape(R)[1])
    if not S:
        hi = np.zeros(shape)
        lo = np.zeros(shape)
    elif exact:
        hi, lo = recombine_exact(S, eL, eR, shape)
    else:
        hi, lo = recombine_dd(S, eL, eR, shape)
    return dict(hi=hi, lo=lo, S=S, dL=dL, dR=dR, eL=eL, eR=eR, pairs=pairs)


def ozaki_gemm(A, B, k, mode="full", exact=False):
    """C = A B with k digit planes per operand; mode 'full' (k^2 products) or
    'triangular' (r + s <= k + 1, k(k+1)/2 products).  FP64 result RN(C_hi + C_lo).
    """
    T = 2 * k if mode == "full" else k + 1
    out = ozaki_product(A, B, k, k, T, exact=exact)
    return out["hi"] + out["lo"], out
