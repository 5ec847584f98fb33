"""Error-free transformations and double-double (pair) arithmetic, vectorised.

ORACLE: test infrastructure only.

Paper: Sec. 2.2 (Knuth's TwoSum; the pair arithmetic of Lange and Rump that drops
the lower word of one operand). TwoProduct uses Dekker's algorithm with Veltkamp
splitting so that it is exact without a fused multiply-add.
"""
from __future__ import annotations

import numpy as np

_SPLITTER = 134217729.0  # 2^27 + 1


def two_sum(a, b):
    """Sec. 2.2: x = fl(a + b), y = fl((a - (x - z)) + (b - z)) with z = fl(x - a).

    a + b = x + y holds exactly (Knuth).
    """
    x = a + b
    z = x - a
    y = (a - (x - z)) + (b - z)
    return x, y


def fast_two_sum(a, b):
    """x + y = a + b exactly, provided |a| >= |b| (or a = 0)."""
    x = a + b
    y = b - (x - a)
    return x, y


def split(a):
    """Veltkamp split: a = hi + lo, each with at most 26 significant bits."""
    c = _SPLITTER * a
    hi = c - (c - a)
    lo = a - hi
    return hi, lo


def two_prod(a, b):
    """Dekker: p = fl(a * b), e = a * b - p exactly (no overflow assumed)."""
    p = a * b
    ah, al = split(a)
    bh, bl = split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def pair_add(a, bh, bl):
    """Sec. 2.2 pair arithmetic: a + (b_h + b_l) ~= c_h + c_l.

    [c_h, t] = TwoSum(a, b_h); c_l = fl(b_l + t).
    """
    ch, t = two_sum(a, bh)
    cl = bl + t
    return ch, cl


def dd_add(ah, al, bh, bl):
    """(ah + al) + (bh + bl) as a normalised double-double (accurate form)."""
    sh, se = two_sum(ah, bh)
    th, te = two_sum(al, bl)
    se = se + th
    sh, se = fast_two_sum(sh, se)
    se = se + te
    return fast_two_sum(sh, se)


def dd_add_d(ah, al, b):
    """(ah + al) + b as a normalised double-double."""
    sh, se = two_sum(ah, b)
    se = se + al
    return fast_two_sum(sh, se)


def dd_mul_d(ah, al, b):
    """(ah + al) * b as a normalised double-double."""
    ph, pe = two_prod(ah, b)
    pe = pe + al * b
    return fast_two_sum(ph, pe)


def dd_div_dd(ah, al, bh, bl):
    """(ah + al) / (bh + bl) to double-double accuracy (one Newton correction)."""
    q1 = ah / bh
    # r = a - q1 * b
    ph, pl = dd_mul_d(bh, bl, q1)
    rh, rl = dd_add(ah, al, -ph, -pl)
    q2 = rh / bh
    return fast_two_sum(q1, q2)


def dd_sum(h, l, axis):
    """Sum of a double-double array along ``axis`` (sequential TwoSum chain)."""
    h = np.moveaxis(np.asarray(h, dtype=np.float64), axis, 0)
    l = np.moveaxis(np.asarray(l, dtype=np.float64), axis, 0)
    sh = np.zeros(h.shape[1:])
    sl = np.zeros(h.shape[1:])
    for k in range(h.shape[0]):
        sh, sl = dd_add(sh, sl, h[k], l[k])
    return sh, sl


def dd_matmul(Lh, Ll, Rh, Rl):
    """Product of two double-double matrices, to about 2^-100 relative accuracy.

    Each term L[i,k] R[k,j] is formed by TwoProduct of the high words plus the
    cross terms in FP64, and accumulated with TwoSum along k (Dot2-style).
    ``Ll`` or ``Rl`` may be None for an FP64 operand.
    """
    Lh = np.asarray(Lh, dtype=np.float64)
    Rh = np.asarray(Rh, dtype=np.float64)
    m, K = Lh.shape
    K2, n = Rh.shape
    assert K == K2
    sh = np.zeros((m, n))
    sl = np.zeros((m, n))
    for k in range(K):
        a = Lh[:, k:k + 1]
        b = Rh[k:k + 1, :]
        p, e = two_prod(a, b)
        if Rl is not None:
            e = e + a * Rl[k:k + 1, :]
        if Ll is not None:
            e = e + Ll[:, k:k + 1] * b
        sh, t = two_sum(sh, p)
        sl = sl + (t + e)
        sh, sl = fast_two_sum(sh, sl)
    return sh, sl
