"""Comparator: the same refinement with native FP64 products (cuBLAS DGEMM via torch).

This is the paper's own formulation run on the GPU with library DGEMM, used by
``bench.py`` as the "native-FP64 refinement" the Ozaki path is measured against.
It is not part of the frx product path and shares no code with it.

Per iteration (Algorithm 1 with Sec. 3 and the Sec. 4.1 parameters):
  beta, alpha  eq. proposed_beta with floor rounding and ceil(log2 sqrt n) (Sec. 4.1), the
               error model's xi as in the frx plan (1 by default; xi <= 0: n, the
               "n delta" of the Sec. 4.1 experiments), from the previous estimates; beta is
               raised where needed so that alpha <= 52 (every FP64 slice keeps a bit);
  X1           fl((tau_j + x) - tau_j) (eq. tau, eq. x);
  A slices     eq. sigma / eq. a with alpha and a rescan of the residual's row maxima,
               n_A - 1 slices plus the remainder (eq. mat_mul);
  V            sum of the n_A FP64 products fl(A^(r) X1), accumulated in double-double;
  r, lambda    double-double column sums;
  W = X1^T (V - X1 D) and X1 E~   plain FP64 products (the paper's "+2");
  X            fl(X1 + X1 E~).
n_A is chosen so that the slices capture as many bits of A as the Ozaki path's
k_V digit planes (8 k_V bits), the product count the paper sweeps by hand.
"""
from __future__ import annotations

import math

import torch

U = 2.0 ** -53


def _two_sum(a, b):
    x = a + b
    z = x - a
    return x, (a - (x - z)) + (b - z)


def _split(a):
    c = 134217729.0 * a
    hi = c - (c - a)
    return hi, a - hi


def _two_prod(a, b):
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def _dd_add(ah, al, bh, bl):
    sh, se = _two_sum(ah, bh)
    th, te = _two_sum(al, bl)
    se = se + th
    x = sh + se
    se = se - (x - sh)
    sh = x
    se = se + te
    x = sh + se
    return x, se - (x - sh)


def _dd_colsum(h, l):
    """Double-double sum over dim 0 by a pairwise tree of accurate additions."""
    while h.shape[0] > 1:
        if h.shape[0] % 2:
            z = torch.zeros_like(h[:1])
            h = torch.cat([h, z])
            l = torch.cat([l, z])
        h, l = _dd_add(h[0::2], l[0::2], h[1::2], l[1::2])
    return h[0], l[0]


def _ceil_log2(m):
    fr, ex = torch.frexp(m)
    return torch.where(fr == 0.5, ex - 1, ex)


def _pow2(e):
    return torch.ldexp(torch.ones_like(e, dtype=torch.float64), e)


def _ceil_log2_sqrt(n):
    return ((n - 1).bit_length() + 1) // 2


def _slices_for(n, eL, eR, tau, kcap=16):
    # the digit-plane count the frx plan gives its V product (8-bit planes, 16 n 2^(eL+eR-8k) <= tau)
    for k in range(1, kcap + 1):
        if math.ldexp(tau, 8 * k - eL - eR - 4) >= float(n):
            return k
    return kcap


def _min_gap(lam):
    s = torch.sort(lam).values
    g = s[1:] - s[:-1]
    g = g[g > 0]
    Lam = float(lam.abs().max())
    return (float(g.min()) if g.numel() else Lam), Lam


def step(A, X, lam_prev, delta, xi=1.0):
    n = X.shape[0]
    g, Lam = _min_gap(lam_prev)
    f = _ceil_log2(X.abs().amax(dim=0))
    S2 = float(torch.sum(_pow2(2 * f)))
    xi = xi if xi > 0 else float(n)
    q = math.sqrt((xi * delta * g) / (Lam * S2)) / (0.75 * U)
    beta = min(max(math.frexp(q)[1] - 1, 3), 47)
    # the FP64 slices of eq. sigma carry 53 - alpha bits: keep at least one (alpha <= 52) by
    # raising beta where a tight target and small gaps would push alpha to 53 or beyond
    beta = max(beta, _ceil_log2_sqrt(n) + 1)
    alpha = 53 - beta + _ceil_log2_sqrt(n)
    tau = 0.75 * _pow2(f + beta)
    X1 = (tau[None, :] + X) - tau[None, :]
    eA = int(_ceil_log2(A.abs().amax(dim=1)).max())
    kV = _slices_for(n, eA, int(f.max()), delta * g)
    bits = 53 - alpha
    nA = max(2, 1 + math.ceil((8 * kV - 53) / bits))
    # V = sum_r fl(A^(r) X1) (eq. mat_mul), accumulated in double-double
    res = A.clone()
    Vh = torch.zeros_like(X)
    Vl = torch.zeros_like(X)
    for r in range(nA):
        if r < nA - 1:
            v = res.abs().amax(dim=1)
            sig = torch.where(v > 0, 0.75 * _pow2(_ceil_log2(v) + alpha), torch.zeros_like(v))[:, None]
            Ar = (sig + res) - sig
            res = res - Ar
        else:
            Ar = res
        P = Ar @ X1
        Vh, e = _two_sum(Vh, P)
        Vl = Vl + e
    # r, lambda, Res and W (Alg. 1)
    ph, pl = _two_prod(X1, X1)
    nh, nl = _dd_colsum(ph, pl)
    qh, ql = _two_prod(X1, Vh)
    dh, dl = _dd_colsum(qh, ql + X1 * Vl)
    q1 = dh / nh
    mh, ml = _two_prod(nh, q1)
    rh, _ = _dd_add(dh, dl, -mh, -(ml + nl * q1))
    lam = q1 + rh / nh
    r = _dd_add(-nh, -nl, torch.ones_like(nh), torch.zeros_like(nh))[0]
    mh, ml = _two_prod(X1, lam[None, :])
    Res = _dd_add(Vh, Vl, -mh, -ml)[0]
    W = X1.T @ Res
    diff = lam[None, :] - lam[:, None]
    eye = torch.eye(n, dtype=torch.bool, device=X.device)
    E = torch.where(eye, (r / 2)[None, :].expand(n, n), W / torch.where(eye, torch.ones_like(diff), diff))
    Xn = X1 + X1 @ E
    stp = float(torch.linalg.norm(Xn - X))
    g2, Lam2 = _min_gap(lam)
    est = stp * stp * Lam2 / (n * g2)
    return Xn, lam, dict(beta=beta, alpha=alpha, nA=nA, products=nA + 2, step=stp, est=est)


def refine(A, X, D, delta, max_iter=10, xi=1.0):
    """Returns (X, lam, info); A, X, D float64 CUDA tensors (X, D are not modified)."""
    lam = D.clone()
    prev = None
    noncontract = 0
    status, it, total, est = "max_iter", 0, 0, math.inf
    for it in range(1, max_iter + 1):
        X, lam, info = step(A, X, lam, delta, xi)
        total += info["products"]
        est = info["est"]
        noncontract = noncontract + 1 if (prev is not None and info["step"] > 0.5 * prev) else 0
        if est <= delta:
            status = "converged"
            break
        if noncontract >= 2:
            status = "stagnated"
            break
        prev = info["step"]
    return X, lam, dict(status=status, iters=it, products=total, err_est=est, nA=info["nA"])
