"""Seeded synthetic inputs for the eigenvector-refinement workloads.

This module builds test matrices and starting guesses only. It holds none of the
refinement method's arithmetic (no slicing, no products of the method, no
correction formula), so both the CPU oracle and the CUDA path can take their
inputs from it without sharing any of the method's code.

Workloads (stand-ins for MATLAB's ``gallery('randsvd', n, -cnd, 3, ...)`` used in
Sec. 4, whose test matrices are symmetric with a geometric spectrum):

* ``spectrum``: geometric eigenvalues lambda_i = cond^(-(n-1-i)/(n-1)), ascending
  from 1/cond to 1; variants ``indefinite`` (seeded random signs) and
  ``clustered`` (pairs lambda_{2m+1} = lambda_{2m}(1 + gap)).
* ``householder_q``: Q = H_1 H_2 ... H_n with H_k = I - 2 v_k v_k^T / (v_k^T v_k)
  and v_k ~ N(0, I), applied in blocks (compact WY form) for speed.
* ``symmetric_matrix``: A = Q diag(lambda) Q^T in FP64, made exactly symmetric by
  mirroring the upper triangle.
* ``initial_guess``: X0 = Q + noise of 2-norm about ``rel``, re-orthonormalised
  by a Householder QR in FP64 (column signs kept), D0 = lambda (1 + rel N(0,1)).
* ``gemm_operand``: entries N(0,1) * exp(phi N(0,1)) (growing exponent spread).

Seeds follow 2602190900 + 1000 * workload + case.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 2602190900


def seed_for(workload: int, case: int = 0) -> int:
    return SEED_BASE + 1000 * workload + case


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def spectrum(n: int, cond: float, variant: str = "spd", seed: int = 0,
             cluster_pairs: int = 16, cluster_gap: float = 1e-10) -> np.ndarray:
    """Ascending geometric spectrum from 1/cond to 1 (randsvd mode 3 shape)."""
    if n == 1:
        lam = np.ones(1)
    else:
        i = np.arange(n, dtype=np.float64)
        lam = cond ** (-(n - 1 - i) / (n - 1))
    if variant == "indefinite":
        s = rng(seed + 7).integers(0, 2, size=n) * 2 - 1
        lam = lam * s
        lam = np.sort(lam)
    elif variant == "clustered":
        lam = lam.copy()
        # spread the pairs over the spectrum: pair m uses indices (2m', 2m'+1)
        m = min(cluster_pairs, n // 2)
        starts = np.linspace(0, n - 2, m).astype(np.int64) // 2 * 2
        for s0 in starts:
            lam[s0 + 1] = lam[s0] * (1.0 + cluster_gap)
        lam = np.sort(lam)
    elif variant != "spd":
        raise ValueError(f"unknown spectrum variant {variant!r}")
    return lam


def householder_q(n: int, seed: int, block: int = 64) -> np.ndarray:
    """Q = H_1 H_2 ... H_n from Gaussian Householder vectors (FP64)."""
    g = rng(seed)
    V = g.standard_normal((n, n))
    Q = np.eye(n)
    for b0 in range(0, n, block):
        Vb = V[:, b0:b0 + block]
        nb = Vb.shape[1]
        tau = 2.0 / np.einsum("ij,ij->j", Vb, Vb)
        # H_1...H_b = I - Vb T Vb^T with T upper triangular (forward accumulation)
        T = np.zeros((nb, nb))
        for k in range(nb):
            T[k, k] = tau[k]
            if k:
                T[:k, k] = -tau[k] * (T[:k, :k] @ (Vb[:, :k].T @ Vb[:, k]))
        Q = Q - ((Q @ Vb) @ T) @ Vb.T
    return Q


def symmetric_matrix(n: int, cond: float, seed: int, variant: str = "spd", **kw):
    """(A, Q, lam): exactly symmetric FP64 A close to Q diag(lam) Q^T."""
    lam = spectrum(n, cond, variant, seed, **kw)
    Q = householder_q(n, seed)
    A = (Q * lam) @ Q.T
    A = np.triu(A) + np.triu(A, 1).T
    return np.ascontiguousarray(A), Q, lam


def initial_guess(Q: np.ndarray, lam: np.ndarray, seed: int, rel: float = 1e-8):
    """(X0, D0): perturbed and re-orthonormalised starting eigenpairs."""
    n = Q.shape[0]
    g = rng(seed + 1)
    noise = g.standard_normal((n, n)) * (rel / (2.0 * np.sqrt(n)))
    Y = Q + noise
    Qr, R = np.linalg.qr(Y)
    X0 = Qr * np.sign(np.diag(R))
    D0 = lam * (1.0 + rel * g.standard_normal(n))
    return np.ascontiguousarray(X0), D0


def gemm_operand(m: int, n: int, phi: float, seed: int) -> np.ndarray:
    g = rng(seed)
    return g.standard_normal((m, n)) * np.exp(phi * g.standard_normal((m, n)))


def workload0():
    """n=64, cond 1e8 SPD, start perturbed by 1e-8, 8 planes of A, delta 1e-14."""
    s = seed_for(0)
    A, Q, lam = symmetric_matrix(64, 1e8, s)
    X0, D0 = initial_guess(Q, lam, s)
    return A, X0, D0


def refine_workload(n: int, cond: float, variant: str = "spd", case: int = 0, rel: float = 1e-8):
    """Full-refinement input: (A, X0, D0, lam)."""
    s = seed_for(2, case)
    A, Q, lam = symmetric_matrix(n, cond, s, variant)
    X0, D0 = initial_guess(Q, lam, s, rel)
    return A, X0, D0, lam


def batched_sizes(count: int = 256, lo: int = 32, hi: int = 512, case: int = 0):
    g = rng(seed_for(3, case))
    n = g.integers(lo, hi + 1, size=count)
    logc = g.uniform(2.0, 12.0, size=count)
    return n, 10.0 ** logc


def _fwht_rows(M):
    """Unnormalised Sylvester-Hadamard transform of every row (exact for integer input)."""
    n = M.shape[1]
    M = M.copy()
    h = 1
    while h < n:
        M = M.reshape(M.shape[0], -1, 2 * h)
        a = M[:, :, :h].copy()
        b = M[:, :, h:].copy()
        M[:, :, :h] = a + b
        M[:, :, h:] = a - b
        M = M.reshape(M.shape[0], n)
        h *= 2
    return M


def _inv_sqrt_dd(n: int):
    """1/sqrt(n) for n = 2^p as a double-double (exact when p is even)."""
    import decimal
    p = n.bit_length() - 1
    with decimal.localcontext() as ctx:
        ctx.prec = 60
        v = decimal.Decimal(1) / decimal.Decimal(n).sqrt()
        hi = float(v)
        lo = float(v - decimal.Decimal(hi))
    if p % 2 == 0:
        assert lo == 0.0
    return hi, lo


def _scaled_dd(num: int, n: int, den: int = 1):
    """num / (den sqrt(n)) for n = 2^p as a double-double."""
    import decimal
    with decimal.localcontext() as ctx:
        ctx.prec = 60
        v = decimal.Decimal(num) / (decimal.Decimal(den) * decimal.Decimal(n).sqrt())
        hi = float(v)
        lo = float(v - decimal.Decimal(hi))
    return hi, lo


def rotated_hadamard_workload(n: int, cond: float, seed: int, rel: float = 1e-8, variant: str = "spd"):
    """Exact-truth workload for n = 2^p whose eigenvectors are not dyadic at any p.

    Columns k and k + n/2 of the Sylvester Hadamard matrix H are rotated by the exact rotation
    R5 / 5, R5 = [[3, -4], [4, 3]]: Q = H R / sqrt(n) with R block-diagonal in those pairs, so
    every entry of Q is +-7 / (5 sqrt n) or +-1 / (5 sqrt n) (not an FP64 number).  With m_k
    distinct positive integers (the geometric magnitudes of ``spectrum(n, cond)`` scaled by 2^S
    and made distinct, as in ``hadamard_workload``) and s_k = +1 or seeded signs, the block
    matrix M = R5 diag(s m) R5^T is an integer matrix, A = H M H 2^-S / n has exact FP64
    entries (|sum| <= 49 sum m < 2^53), and A (H R5) = 25 (H R5) diag(s m) 2^-S exactly: the
    eigenpairs of the stored A are lam_k = 25 s_k m_k 2^-S and the columns of Q.
    Returns (A, X0, D0, lam, Qh, Ql, info) like ``hadamard_workload``.
    """
    p = n.bit_length() - 1
    if n < 2 or (1 << p) != n:
        raise ValueError("n must be a power of 2")
    geom = spectrum(n, cond)
    S = int(np.floor(np.log2(2.0 ** 52 / (49.0 * float(np.sum(geom))))))
    m = np.maximum(np.rint(geom * 2.0 ** S), 1).astype(np.int64)
    k = np.arange(n, dtype=np.int64)
    m = np.maximum.accumulate(m - k) + k                     # strictly increasing
    assert 49 * int(np.sum(m)) < (1 << 53)
    if variant == "indefinite":
        sgn = rng(seed + 7).integers(0, 2, size=n).astype(np.int64) * 2 - 1
    elif variant == "spd":
        sgn = np.ones(n, dtype=np.int64)
    else:
        raise ValueError(f"unknown variant {variant!r}")
    # eigenvalue index j of H-column pair (a, a + n/2): a seeded assignment of the sorted
    # magnitudes to the columns, so that each rotated pair mixes two unrelated eigenvalues
    perm = rng(seed + 3).permutation(n)
    sm = (sgn * m)[perm]                                     # s m of H-column k
    h = n // 2
    a, b = sm[:h], sm[h:]
    M = np.zeros((n, n), dtype=np.int64)
    idx = np.arange(h)
    M[idx, idx] = 9 * a + 16 * b
    M[idx + h, idx + h] = 16 * a + 9 * b
    M[idx, idx + h] = 12 * (a - b)
    M[idx + h, idx] = 12 * (a - b)
    W = _fwht_rows(M)                                        # M H
    W = _fwht_rows(np.ascontiguousarray(W.T)).T              # H M H
    A = np.ascontiguousarray(W.astype(np.float64) * (2.0 ** -S / n))
    del W, M
    lam_all = 25.0 * sm.astype(np.float64) * 2.0 ** -S
    order = np.argsort(lam_all, kind="stable")
    lam = lam_all[order]
    # H R5: column k (k < n/2) = 3 h_k + 4 h_{k+n/2}, column k + n/2 = -4 h_k + 3 h_{k+n/2}
    Hm = _fwht_rows(np.eye(n, dtype=np.int64))
    HR = np.empty((n, n), dtype=np.int64)
    HR[:, :h] = 3 * Hm[:, :h] + 4 * Hm[:, h:]
    HR[:, h:] = -4 * Hm[:, :h] + 3 * Hm[:, h:]
    del Hm
    HR = HR[:, order]
    Qh = np.empty((n, n))
    Ql = np.empty((n, n))
    for v in (7, 1, -1, -7):
        hi, lo = _scaled_dd(v, n, 5)
        sel = HR == v
        Qh[sel] = hi
        Ql[sel] = lo
    assert np.all(np.isin(HR, (7, 1, -1, -7)))
    del HR
    g = rng(seed + 1)
    Y = Qh + g.standard_normal((n, n)) * (rel / (2.0 * np.sqrt(n)))
    Qr, R = np.linalg.qr(Y)
    X0 = np.ascontiguousarray(Qr * np.sign(np.diag(R)))
    D0 = lam * (1.0 + rel * g.standard_normal(n))
    gaps = np.diff(lam)
    info = dict(scale_exp=-S, min_gap=float(gaps.min()), max_abs=float(np.abs(lam).max()),
                cond=float(np.abs(lam).max() / np.abs(lam).min()))
    return A, X0, D0, lam, Qh, Ql, info


def hadamard_workload(n: int, cond: float, seed: int, rel: float = 1e-8, variant: str = "spd"):
    """Exact-truth workload for n = 2^p.

    A = H diag(s_k m_k) H 2^-S / n with H the Sylvester Hadamard matrix, m_k distinct positive
    integers and s_k = +1 ("spd") or seeded random signs ("indefinite").  Every entry of A is
    an exact FP64 number (|sum_k +-m_k| < 2^53, power-of-two scaling), so the eigenvectors of
    the stored A are exactly the columns of H / sqrt(n).  The magnitudes follow the geometric
    spectrum of ``spectrum(n, cond)``: m_k = round(2^S geom_k) with S as large as the 2^53
    bound allows, raised where needed to keep the m_k distinct (for cond * n large the
    smallest eigenvalues become consecutive integers, widening the smallest gaps).
    Returns (A, X0, D0, lam, Qh, Ql, info): lam ascending, Q = Qh + Ql = H / sqrt(n) with
    columns ordered like lam (Ql = 0 when p is even); X0, D0 as in ``initial_guess``.
    """
    p = n.bit_length() - 1
    if n < 2 or (1 << p) != n:
        raise ValueError("n must be a power of 2")
    geom = spectrum(n, cond)
    S = int(np.floor(np.log2(2.0 ** 52 / float(np.sum(geom)))))
    m = np.maximum(np.rint(geom * 2.0 ** S), 1).astype(np.int64)
    k = np.arange(n, dtype=np.int64)
    m = np.maximum.accumulate(m - k) + k                     # strictly increasing
    assert int(np.sum(m)) < (1 << 53)
    if variant == "indefinite":
        sgn = rng(seed + 7).integers(0, 2, size=n).astype(np.int64) * 2 - 1
    elif variant == "spd":
        sgn = np.ones(n, dtype=np.int64)
    else:
        raise ValueError(f"unknown variant {variant!r}")
    sm = sgn * m
    W = _fwht_rows(np.diag(sm))                              # diag(sm) H
    W = _fwht_rows(np.ascontiguousarray(W.T)).T              # H diag(sm) H
    A = np.ascontiguousarray(W.astype(np.float64) * (2.0 ** -S / n))
    del W
    lam_all = sm.astype(np.float64) * 2.0 ** -S
    order = np.argsort(lam_all, kind="stable")
    lam = lam_all[order]
    Hm = _fwht_rows(np.eye(n, dtype=np.int8).astype(np.int64)[:, :])   # H (symmetric)
    Hc = Hm[:, order].astype(np.float64)
    del Hm
    ih, il = _inv_sqrt_dd(n)
    Qh = np.ascontiguousarray(Hc * ih)
    Ql = np.ascontiguousarray(Hc * il)
    g = rng(seed + 1)
    Y = Qh + g.standard_normal((n, n)) * (rel / (2.0 * np.sqrt(n)))
    Qr, R = np.linalg.qr(Y)
    X0 = np.ascontiguousarray(Qr * np.sign(np.diag(R)))
    D0 = lam * (1.0 + rel * g.standard_normal(n))
    gaps = np.diff(lam)
    info = dict(scale_exp=-S, min_gap=float(gaps.min()), max_abs=float(np.abs(lam).max()),
                cond=float(np.abs(lam).max() / np.abs(lam).min()))
    return A, X0, D0, lam, Qh, Ql, info


def banded_workload(n: int, bw: int, seed: int, rel: float = 1e-8):
    """Sparse stand-in (the paper's ELSES matrices are not available): a symmetric band matrix
    with half-bandwidth bw (k = 2 bw + 1 nonzeros in an interior row), entries N(0, 1) inside
    the band, exactly symmetric.  The start is its FP64 eigenvector basis (numpy eigh) perturbed
    by `rel` and re-orthonormalised, as in ``initial_guess``.  Returns (A, X0, D0, lam)."""
    g = rng(seed)
    A = np.zeros((n, n))
    for d in range(bw + 1):
        v = g.standard_normal(n - d)
        A[np.arange(n - d), np.arange(d, n)] = v
        A[np.arange(d, n), np.arange(n - d)] = v
    lam, Q = np.linalg.eigh(A)
    X0, D0 = initial_guess(Q, lam, seed, rel)
    return np.ascontiguousarray(A), X0, D0, lam


def random_sparse_workload(n: int, per_row: int, seed: int, rel: float = 1e-8):
    """Sparse stand-in with an irregular pattern: a symmetric matrix whose row i holds
    per_row / 2 entries N(0, 1) at seeded random columns, mirrored (about per_row nonzeros per
    row), and a diagonal N(0, 1) + 4.  The start is its FP64 eigenvector basis (numpy eigh)
    perturbed by `rel` and re-orthonormalised.  Returns (A, X0, D0, lam)."""
    g = rng(seed)
    A = np.zeros((n, n))
    for i in range(n):
        cols = g.choice(n, per_row // 2, replace=False)
        v = g.standard_normal(cols.size)
        A[i, cols] = v
        A[cols, i] = v
    A[np.arange(n), np.arange(n)] = g.standard_normal(n) + 4.0
    lam, Q = np.linalg.eigh(A)
    X0, D0 = initial_guess(Q, lam, seed, rel)
    return np.ascontiguousarray(A), X0, D0, lam
