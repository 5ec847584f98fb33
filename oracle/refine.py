"""Forward-error-oriented Ogita-Aishima refinement, step by step (Alg. 1 + Sec. 3-4.1).

ORACLE: test infrastructure only.

One iteration (Algorithm 1 with the Sec. 3 modification, eq. mat_mul):
  plan   beta from eq. proposed_beta with floor rounding (Sec. 4.1) and the error
         model's xi = 1 by default (xi = n, the "n delta" of the Sec. 4.1 experiments,
         is an option), alpha = 53 - beta + ceil(log2 sqrt n) (Sec. 4.1), using the
         previous eigenvalue estimates (the circularity is broken by lagging them);
  X1     = fl((tau_j + x_ij) - tau_j), tau_j = 0.75 2^ceil(log2 w_j) 2^beta (eq. tau, x);
  V      = accurate A X1 from exact 8-bit digit-plane products (eq. mat_mul);
  r_i    = 1 - x1_i^T x1_i                                            (Alg. 1);
  lam_i  = x1_i^T v_i / (1 - r_i)                                     (Alg. 1);
  W      = X1^T (V - X1 diag(lam))                                    (Alg. 1);
  E~_ij  = w_ij / (lam_j - lam_i) (i != j), r_i / 2 (i = j)           (Alg. 1);
  X      <- RN(X1 + X1 E~) by pair arithmetic                         (Alg. 1, Sec. 2.2).

Readings where the paper is silent (each also listed in the design notes):
* digit planes: 8-bit digits on a fixed grid (see ``ozaki``); X1 is exactly the
  first s_X = ceil((54 - beta) / 8) planes' worth of bits, so V's products are
  all exact and only the truncation of A to k_V planes (and of the pair set to
  r + s <= k_V + 1) is approximate;
* slice counts (the paper sweeps n_A by hand): k = smallest k with
  16 n 2^(eL + eR - 8k) <= tau, evaluated exactly as 2^(8k - eL - eR - 4) tau >= n,
  where eL, eR are the operands' largest exponents and tau = delta * g for V and W,
  delta for the update product.  Every entry of the dropped part is a sum over n
  terms of digit tails below 2^(eL + eR - 8k); taking such sums to grow like sqrt(n)
  (the reading Sec. 4.1 itself makes when it replaces log2 n by ceil(log2 sqrt n)),
  and the 2-norm of an n x n matrix of such entries like sqrt(n) times their size,
  gives n 2^(eL + eR - 8k); the factor 16 is the margin, calibrated on randsvd-like
  and exact-truth matrices where a factor 1 already leaves the forward error
  unchanged;  a fixed k_V may be forced (``slices_A``);
* the slice products' exact int32 sums need pairs * n * 2^14 < 2^31: the update
  product (up to k_U pairs per anti-diagonal) takes at most floor((2^17 - 1) / n)
  planes (16 for n < 8192); V's and W's pairs are at most s_X <= 7;
* beta is clamped to [3, 47] (tau-trick valid, X1 keeps at least one plane);
* stopping test: ||E~|| cannot fall below ||X^(2)|| (every step re-corrects the
  truncated tail), so the test uses the observed step d_k = ||X_k - X_{k-1}||_F:
  est_k = d_k^2 * Lam / (xi_stop * g) with xi_stop = n (the Sec. 4.1 calibration
  xi = n of the error model eq. assume2); converged when est_k <= delta;
  'stagnated' when d_k > d_{k-1} / 2 for k >= 2 without convergence;
* clusters (excluded by the paper): pairs with |lam_j - lam_i| <= omega take
  e~_ij = r_ij / 2 with r_ij = -x1_i^T x1_j, the Ogita-Aishima rule; omega = 0 by
  default (only equal estimates), or 'auto': omega = 2 (||W||_F + Lam ||diag R||_2).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import ddarith as dd
from . import ozaki as oz

U = 2.0 ** -53


@dataclasses.dataclass
class Options:
    slices_A: int = 0            # 0: automatic k_V; >0: fixed number of A planes
    xi: float | None = 1.0       # eq. proposed_beta's xi; None: xi = n (the Sec. 4.1 "n delta")
    beta_rounding: str = "floor"  # Sec. 4.1 floor; "ceil" = eq. proposed_beta
    theory_alpha: bool = False   # alpha = ceil(53 + log2 n - beta) instead of Sec. 4.1
    beta_override: int | None = None
    k_cap: int = 16
    max_iter: int = 10
    xi_stop: float | None = None  # None: n
    cluster: object = 0.0        # threshold omega (float) or "auto"
    x_planes: int = 0            # > 0: X kept at x_planes digit planes, no truncation rule
                                 # (the "previous study" of Sec. 4: both operands sliced)
    sparse_rule: bool = False    # the sparse-matrix rule of Sec. 4: beta with min(k, sqrt n)
                                 # in place of sqrt n, alpha with ceil(log2 k); k = max row nnz


def ceil_log2_sqrt(n: int) -> int:
    """ceil(log2 sqrt n) for integer n >= 1, exactly."""
    return ((n - 1).bit_length() + 1) // 2


def ceil_log2_int(n: int) -> int:
    return (n - 1).bit_length()


def floor_log2(x: float) -> int:
    fr, ex = math.frexp(x)
    return ex - 1


def ceil_log2f(x: float) -> int:
    fr, ex = math.frexp(x)
    return ex - 1 if fr == 0.5 else ex


def min_gap(lam, omega=0.0):
    """Smallest |lam_j - lam_i| over adjacent sorted estimates exceeding omega.

    Returns (g, Lam); g = Lam if no gap exceeds omega (or n == 1).
    """
    lam = np.asarray(lam, dtype=np.float64)
    Lam = float(np.max(np.abs(lam)))
    s = np.sort(lam)
    gaps = s[1:] - s[:-1]
    gaps = gaps[gaps > omega]
    g = float(np.min(gaps)) if gaps.size else Lam
    return g, Lam


def beta_rule(n, delta, g, Lam, S2, opts: Options) -> int:
    """Sec. 4.1: beta = floor(log2((1/(0.75u)) sqrt(n delta g / (Lam sum_j 2^(2f_j)))))."""
    if opts.beta_override is not None:
        return int(opts.beta_override)
    xi = float(n) if opts.xi is None else float(opts.xi)
    if g <= 0.0 or Lam <= 0.0 or S2 <= 0.0:
        return 3
    q = math.sqrt((xi * delta * g) / (Lam * S2)) / (0.75 * U)
    b = floor_log2(q) if opts.beta_rounding == "floor" else ceil_log2f(q)
    return int(min(max(b, 3), 47))


def alpha_rule(n, beta, opts: Options) -> int:
    if opts.theory_alpha:
        return 53 - beta + ceil_log2_int(n)
    return 53 - beta + ceil_log2_sqrt(n)


SLICE_MARGIN_LOG2 = 4   # the factor 16 of the slice rule


def slices_for(n, eL, eR, tau, k_cap):
    """Smallest k >= 1 with 16 n 2^(eL + eR - 8k) <= tau, i.e. 2^(8k - eL - eR - 4) tau >= n
    (ldexp is exact), capped at k_cap; 0 when an operand is zero."""
    if eL == oz.EZERO or eR == oz.EZERO:
        return 0
    for k in range(1, k_cap + 1):
        if math.ldexp(tau, oz.DIGIT_BITS * k - int(eL) - int(eR) - SLICE_MARGIN_LOG2) >= float(n):
            return k
    return k_cap


def int32_planes(n):
    """Largest k with k * n * 2^14 < 2^31 (exact int32 sums of up to k pairs of products
    of two 8-bit digits over n terms)."""
    return (2 ** 31 - 1) // (n * oz.DIGIT_MAX * oz.DIGIT_MAX)


def sum_pow4(f):
    """sum_j 2^(2 f_j) over nonzero columns, exactly rounded (math.fsum)."""
    return math.fsum(math.ldexp(1.0, 2 * int(x)) for x in f if x != oz.EZERO)


def plan(A, X, lam_prev, delta, opts: Options, omega_prev=0.0):
    n = X.shape[0]
    f = oz.col_exponents(X)
    g, Lam = min_gap(lam_prev, omega_prev)
    S2 = sum_pow4(f)
    # previous-study form: X represented by x_planes digit planes, i.e. rounded to the grid
    # of plane x_planes, which is the tau grid of beta = 54 - 8 x_planes
    kmax = max(int(np.max(np.count_nonzero(A, axis=1))), 1)
    if opts.x_planes > 0:
        beta = 54 - oz.DIGIT_BITS * opts.x_planes
    elif opts.sparse_rule:
        # Sec. 4 (sparse matrices): gamma min(k, sqrt n) sqrt(1 / S2) / (0.75 u) with
        # gamma = sqrt(delta gap / max|lam|) is the Sec. 4.1 form with xi = min(k, sqrt n)^2
        beta = beta_rule(n, delta, g, Lam, S2, dataclasses.replace(opts, xi=float(min(kmax * kmax, n))))
    else:
        beta = beta_rule(n, delta, g, Lam, S2, opts)
    alpha = 53 - beta + ceil_log2_int(kmax) if opts.sparse_rule else alpha_rule(n, beta, opts)
    sX = -(-(54 - beta) // oz.DIGIT_BITS)
    eA = oz.row_exponents(A)
    eAmax = int(np.max(eA))
    fmax = int(np.max(f))
    if opts.slices_A > 0:
        kV = int(opts.slices_A)
    else:
        kV = slices_for(n, eAmax, fmax, delta * g, opts.k_cap)
    return dict(n=n, f=f, g=g, Lam=Lam, S2=S2, beta=beta, alpha=alpha, sX=sX,
                eA=eA, kV=kV)


def step(A, X, lam_prev, delta, opts: Options | None = None, omega_prev=0.0, exact=False):
    """One iteration. Returns (X_new, lam, info)."""
    opts = opts or Options()
    A = np.asarray(A, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    p = plan(A, X, lam_prev, delta, opts, omega_prev)
    beta, sX, kV, f, eA = p["beta"], p["sX"], p["kV"], p["f"], p["eA"]

    # X^(1) (eq. tau, eq. x) and V = A X^(1) (eq. mat_mul)
    if opts.x_planes > 0:
        # the sum of the x_planes digit planes of X (exact: X minus the slicing residual)
        _, _, resid = oz.slice_cols(X, opts.x_planes, f)
        X1 = X - resid
    else:
        X1, _ = oz.tau_truncate_cols(X, beta, f)
    V = oz.ozaki_product(A, X1, kV, sX, kV + 1, eL=eA, eR=f, exact=exact)
    Vh, Vl = V["hi"], V["lo"]

    # r_i = 1 - x_i^T x_i ; lam_i = x_i^T v_i / (1 - r_i)
    ph, pl = dd.two_prod(X1, X1)
    nh, nl = dd.dd_sum(ph, pl, axis=0)            # x_i^T x_i (double-double)
    r = dd.dd_add_d(-nh, -nl, 1.0)[0]
    qh, ql = dd.two_prod(X1, Vh)
    ql = ql + X1 * Vl
    dh, dl = dd.dd_sum(qh, ql, axis=0)            # x_i^T v_i
    lam = dd.dd_div_dd(dh, dl, nh, nl)[0]

    # Res = V - X1 diag(lam) (double-double, then FP64); W = X1^T Res
    mh, ml = dd.two_prod(X1, lam[None, :])
    Res = dd.dd_add(Vh, Vl, -mh, -ml)[0]
    h = oz.col_exponents(Res)
    g = p["g"]
    kW = slices_for(n, int(np.max(f)), int(np.max(h)), delta * g, opts.k_cap)
    if kW > 0:
        Wp = oz.ozaki_product(X1.T, Res, min(sX, kW), kW, kW + 1, eL=f, eR=h, exact=exact)
        W = Wp["hi"] + Wp["lo"]
    else:
        Wp = None
        W = np.zeros((n, n))

    # E~ with the optional cluster rule
    if opts.cluster == "auto":
        offd = W - np.diag(np.diag(W))
        omega = 2.0 * (math.sqrt(float(np.sum(offd * offd))) + p["Lam"] * float(np.linalg.norm(r)))
    else:
        omega = float(opts.cluster)
    diff = lam[None, :] - lam[:, None]            # lam_j - lam_i
    clus = np.abs(diff) <= omega
    np.fill_diagonal(clus, False)
    with np.errstate(divide="ignore", invalid="ignore"):
        E = np.where(clus, 0.0, W / np.where(clus, 1.0, diff))
    if np.any(clus):
        ii, jj = np.nonzero(clus)
        for i, j in zip(ii, jj):
            th, tl = dd.two_prod(X1[:, i], X1[:, j])
            sh, sl = dd.dd_sum(th, tl, axis=0)
            E[i, j] = -sh / 2.0                       # r_ij / 2
    np.fill_diagonal(E, r / 2.0)

    # the update X <- accsum(X1, X1 E~): U = X1 E~ (rows of X1, columns of E~)
    rho = oz.row_exponents(X1)
    eta = oz.col_exponents(E)
    kU = min(slices_for(n, int(np.max(rho)), int(np.max(eta)), delta, opts.k_cap), int32_planes(n))
    if kU > 0:
        Up = oz.ozaki_product(X1, E, kU, kU, kU + 1, eL=rho, eR=eta, exact=exact)
        ch, cl = dd.pair_add(X1, Up["hi"], Up["lo"])
        Xn = ch + cl
    else:
        Up = None
        Xn = X1.copy()

    normE = math.sqrt(float(np.sum(E * E)))
    dX = Xn - X
    step_norm = math.sqrt(float(np.sum(dX * dX)))
    g_new, Lam_new = min_gap(lam, omega)
    xs = float(n) if opts.xi_stop is None else float(opts.xi_stop)
    est = step_norm * step_norm * Lam_new / (xs * g_new) if g_new > 0 else math.inf
    info = dict(plan=p, beta=beta, alpha=p["alpha"], sX=sX, kV=kV, kW=kW, kU=kU,
                products=len(V["pairs"]) + (len(Wp["pairs"]) if Wp else 0) + (len(Up["pairs"]) if Up else 0),
                normE=normE, step=step_norm, est=est, omega=omega, r=r, W=W, E=E, X1=X1, Vh=Vh, Vl=Vl,
                Res=Res, h=h, S_V=V["S"], clustered=int(np.sum(clus)) // 2,
                Uh=Up["hi"] if Up else np.zeros((n, n)), Ul=Up["lo"] if Up else np.zeros((n, n)))
    return Xn, lam, info


def refine(A, X, D, delta, opts: Options | None = None, exact=False, history=None):
    """Iterate until the stopping test passes. Returns (X, lam, info)."""
    opts = opts or Options()
    if not (delta > U):
        raise ValueError("delta must exceed the unit roundoff (Sec. 3.1)")
    lam = np.asarray(D, dtype=np.float64)
    prev_step = None
    noncontract = 0
    omega = 0.0
    status = "max_iter"
    total_products = 0
    it = 0
    est = math.inf
    for it in range(1, opts.max_iter + 1):
        X, lam, info = step(A, X, lam, delta, opts, omega, exact)
        omega = info["omega"]
        total_products += info["products"]
        est = info["est"]
        if history is not None:
            history.append(dict(X=X.copy(), lam=lam.copy(), **{k: info[k] for k in
                                ("beta", "alpha", "sX", "kV", "kW", "kU", "products", "normE", "step", "est")}))
        # stagnation (reading of the missing stopping rule): two consecutive steps that
        # fail to halve; a single one occurs when the start lies outside Theorem 1's basin
        # and the next step repairs the first
        noncontract = noncontract + 1 if (prev_step is not None and info["step"] > 0.5 * prev_step) else 0
        if est <= delta:
            status = "converged"
            break
        if noncontract >= 2:
            status = "stagnated"
            break
        prev_step = info["step"]
    return X, lam, dict(status=status, iters=it, err_est=est, products=total_products)
