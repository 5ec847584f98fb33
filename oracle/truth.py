"""Reference eigenvectors of a stored FP64 matrix and the forward-error metric.

ORACLE: test infrastructure only.

``eigvecs_dd`` refines a starting basis in double-double with the original
Ogita-Aishima iteration written through R and S (Sec. 2.4):
    R = I - X^T X,  S = X^T A X,  lam_i = s_ii / (1 - r_ii),
    e_ij = (s_ij + lam_j r_ij) / (lam_j - lam_i) (i != j),  e_ii = r_ii / 2,
    X <- X + X E,
with every product formed by ``ddarith.dd_matmul``.  It shares no code with the
Alg. 1 / Ozaki oracle in ``refine`` (different formulation, different products),
so agreement between the two is evidence for both.

``forward_error`` is ||X - X^||_2 with X^'s columns sign-aligned to X by the sign
of x_i^T x^_i (the 2-norm, as in Sec. 1 and Sec. 3.1), formed in double-double and
rounded to FP64 before an SVD.
"""
from __future__ import annotations

import math

import numpy as np

from . import ddarith as dd


def eigvecs_dd(A, X0, tol=1e-28, max_iter=12):
    """Returns (Xh, Xl, lam, history of ||E||_F)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    Xh = np.array(X0, dtype=np.float64)
    Xl = np.zeros_like(Xh)
    hist = []
    lam = None
    for _ in range(max_iter):
        Vh, Vl = dd.dd_matmul(A, None, Xh, Xl)
        Gh, Gl = dd.dd_matmul(Xh.T, Xl.T, Xh, Xl)          # X^T X
        Sh, Sl = dd.dd_matmul(Xh.T, Xl.T, Vh, Vl)          # X^T A X
        Rh, Rl = dd.dd_add(np.eye(n), np.zeros((n, n)), -Gh, -Gl)
        rd_h, rd_l = np.diag(Rh).copy(), np.diag(Rl).copy()
        den_h, den_l = dd.dd_add_d(-rd_h, -rd_l, 1.0)
        lam = dd.dd_div_dd(np.diag(Sh).copy(), np.diag(Sl).copy(), den_h, den_l)[0]
        # numerator s_ij + lam_j r_ij (double-double), then divide in FP64
        ph, pl = dd.two_prod(Rh, lam[None, :])
        pl = pl + Rl * lam[None, :]
        nh, nl = dd.dd_add(Sh, Sl, ph, pl)
        diff = lam[None, :] - lam[:, None]
        np.fill_diagonal(diff, 1.0)
        E = (nh + nl) / diff
        np.fill_diagonal(E, (rd_h + rd_l) / 2.0)
        normE = math.sqrt(float(np.sum(E * E)))
        hist.append(normE)
        Ph, Pl = dd.dd_matmul(Xh, Xl, E, None)
        Xh, Xl = dd.dd_add(Xh, Xl, Ph, Pl)
        if normE < tol or (len(hist) > 2 and normE > 0.5 * hist[-2]):
            break
    return Xh, Xl, lam, hist


def forward_error(Xh, Xl, Xhat):
    """||X - X^||_2 with per-column sign alignment (X given as double-double)."""
    Xhat = np.asarray(Xhat, dtype=np.float64)
    s = np.sign(np.einsum("ij,ij->j", Xh, Xhat))
    s[s == 0] = 1.0
    Y = Xhat * s[None, :]
    dh, dl = dd.dd_add(Xh, Xl, -Y, np.zeros_like(Y))
    return float(np.linalg.norm(dh + dl, 2))


def subspace_error(Xh, Xl, Xhat, cols):
    """||sin Theta|| between span(X[:, cols]) and span(X^[:, cols]) (2-norm)."""
    Xt = (Xh + Xl)[:, cols]
    Qt, _ = np.linalg.qr(Xt)
    Qh, _ = np.linalg.qr(np.asarray(Xhat)[:, cols])
    P = Qh - Qt @ (Qt.T @ Qh)
    return float(np.linalg.norm(P, 2))
