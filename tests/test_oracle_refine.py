"""Pins for the refinement oracle (Alg. 1, Sec. 3, Sec. 4.1) and the ground truth."""
import math

import numpy as np
import pytest

from oracle import ddarith as dd
from oracle import ozaki as oz
from oracle import refine as rf
from oracle import truth as tr
from paper_2602_19090_gb300 import synth

U = 2.0 ** -53


def test_beta_alpha_worked_example():
    # Sec. 4.1 rule worked by hand: n = 4096, delta = 1e-14, min gap 2.25e-7, max|lam| = 1,
    # every column maximum in (2^-4, 2^-3] so sum_j 2^(2 f_j) = 4096 * 2^-6 = 64.
    # 4096 * 1e-14 * 2.25e-7 / 64 = 1.44e-19; sqrt = 3.795e-10; / (0.75 * 2^-53) = 4.557e6;
    # log2 = 22.12 -> beta = 22 (floor), 23 (ceil);  alpha = 53 - 22 + ceil(log2 64) = 37
    # (theory: 53 - 22 + log2 4096 = 43);  X^(1) keeps bits 2^f ... 2^(f+22-53):
    # 32 bit positions -> ceil(32 / 8) = 4 planes of 8-bit digits.
    o = rf.Options(xi=None)
    assert rf.beta_rule(4096, 1e-14, 2.25e-7, 1.0, 64.0, o) == 22
    assert rf.beta_rule(4096, 1e-14, 2.25e-7, 1.0, 64.0, rf.Options(xi=None, beta_rounding="ceil")) == 23
    # the default xi = 1 of eq. proposed_beta: 1e-14 * 2.25e-7 / 64 = 3.516e-23; sqrt = 5.930e-12;
    # / (0.75 * 2^-53) = 7.121e4; log2 = 16.12 -> beta = 16 (sqrt 4096 = 2^6 below the n delta form)
    assert rf.beta_rule(4096, 1e-14, 2.25e-7, 1.0, 64.0, rf.Options()) == 16
    assert rf.alpha_rule(4096, 22, o) == 37
    assert rf.alpha_rule(4096, 22, rf.Options(theory_alpha=True)) == 43
    X = np.full((4096, 3), 0.07)
    p = rf.plan(np.eye(3), X[:3], np.array([0.0, 2.25e-7, 1.0]), 1e-14, o)
    assert p["f"].tolist() == [-3, -3, -3]
    assert -(-(54 - 22) // oz.DIGIT_BITS) == 4


def test_ceil_log2_sqrt_exact():
    for n in range(1, 70000):
        c = rf.ceil_log2_sqrt(n)
        assert 4 ** (c - 1) < n <= 4 ** c or (n == 1 and c == 0)


def test_slice_rule_worked_by_hand():
    # 16 n 2^(eL + eR - 8k) <= tau, smallest k:
    #   n = 64, eL = eR = 0, tau = 2^-40: 2^(4 + 6 - 8k) <= 2^-40  <=>  8k >= 50  ->  k = 7
    assert rf.slices_for(64, 0, 0, 2.0 ** -40, 16) == 7
    #   the same with tau = 2^-46: 8k >= 56 -> k = 7 exactly at the boundary; a hair below -> 8
    assert rf.slices_for(64, 0, 0, 2.0 ** -46, 16) == 7
    assert rf.slices_for(64, 0, 0, 2.0 ** -46 * (1 - 2.0 ** -52), 16) == 8
    #   n = 4096, eL = -2, eR = -3, tau = 1e-14 * 2.25e-7 = 2^-68.59: 4 + 12 - 5 - 8k <= -68.59
    #   <=>  8k >= 79.59  ->  k = 10;  with n = 33000 (log2 = 15.01): 8k >= 82.60 -> k = 11
    assert rf.slices_for(4096, -2, -3, 1e-14 * 2.25e-7, 16) == 10
    assert rf.slices_for(33000, -2, -3, 1e-14 * 2.25e-7, 16) == 11
    # a zero operand needs no product; the cap holds
    assert rf.slices_for(64, oz.EZERO, 0, 1e-20, 16) == 0
    assert rf.slices_for(64, 0, 0, 1e-300, 5) == 5


@pytest.mark.parametrize("n,cond,tau", [(128, 1e6, 1e-18), (200, 1e3, 1e-24), (96, 1e10, 1e-21)])
def test_slice_rule_keeps_the_dropped_part_below_tau(n, cond, tau):
    # the rule's promise, measured: A X^(1) with the rule's k planes of A and the pair set
    # r + s <= k + 1 (X^(1), a beta = 20 truncation of eigenvectors, is exact in its 5 planes)
    # differs from the exact product (double-double) by less than tau in the 2-norm
    A, Q, lam = synth.symmetric_matrix(n, cond, 11)
    X1, f = oz.tau_truncate_cols(Q, 20)
    eA = oz.row_exponents(A)
    k = rf.slices_for(n, int(np.max(eA)), int(np.max(f)), tau, 16)
    out = oz.ozaki_product(A, X1, k, 5, k + 1, eL=eA, eR=f)
    Vh, Vl = dd.dd_matmul(A, None, X1, None)
    err = (out["hi"] - Vh) + (out["lo"] - Vl)
    assert np.linalg.norm(err, 2) <= tau
    # and one plane fewer is not always enough: the rule is not vacuous
    out = oz.ozaki_product(A, X1, k - 1, 5, k, eL=eA, eR=f)
    err = (out["hi"] - Vh) + (out["lo"] - Vl)
    assert np.linalg.norm(err, 2) > tau * 2.0 ** -12


def test_w_identity():
    # For i != j, w_ij = s_ij + lam_j r_ij with S = X^T A X, R = I - X^T X (Sec. 2.4).
    A, X0, D0 = synth.workload0()
    delta = 1e-14
    Xn, lam, info = rf.step(A, X0, D0, delta, rf.Options())
    X1 = info["X1"]
    Vh, Vl = dd.dd_matmul(A, None, X1, None)
    Sh, Sl = dd.dd_matmul(X1.T, None, Vh, Vl)
    Gh, Gl = dd.dd_matmul(X1.T, None, X1, None)
    ph, pl = dd.two_prod(-Gh, lam[None, :])
    pl = pl - Gl * lam[None, :]
    rh, rl = dd.dd_add(Sh, Sl, ph, pl)                 # s_ij - (X^T X)_ij lam_j
    ref = rh + rl
    off = ~np.eye(64, dtype=bool)
    err = np.abs(info["W"] - ref)[off]
    g = info["plan"]["g"]
    assert np.sqrt(np.sum(err ** 2)) <= delta * g / 4


def test_diagonal_matrix_fixed_point():
    d = np.array([1.0, -3.0, 0.5, 2.0, 7.0, -0.25])
    A = np.diag(d)
    X = np.eye(6)
    Xn, lam, info = rf.step(A, X, d * (1 + 1e-9), 1e-14, rf.Options())
    assert np.array_equal(Xn, X)
    assert np.array_equal(lam, d)
    assert np.all(info["E"] == 0.0)


def test_reduces_to_classic_ogita_aishima():
    # With X already on the tau grid X^(1) = X, and one step equals the R/S form.
    A, Q, lam = synth.symmetric_matrix(24, 10.0, 77)
    X0, D0 = synth.initial_guess(Q, lam, 77, 1e-6)
    X0 = np.round(X0 * 2.0 ** 28) / 2.0 ** 28
    opts = rf.Options(beta_override=3)
    X1, _ = oz.tau_truncate_cols(X0, 3)
    assert np.array_equal(X1, X0)
    Xn, lam_o, _ = rf.step(A, X0, D0, 1e-15, opts)
    Th, Tl, lam_t, _ = tr.eigvecs_dd(A, X0, max_iter=1)
    assert np.max(np.abs(Xn - (Th + Tl))) <= 4 * U
    assert np.max(np.abs(lam_o - lam_t)) <= 4 * U * np.max(np.abs(lam_t))


def _well_separated(n=16, rel=1e-6, seed=5):
    A, Q, lam = synth.symmetric_matrix(n, 10.0, seed)
    X0, D0 = synth.initial_guess(Q, lam, seed, rel)
    Xh, Xl, lam_t, _ = tr.eigvecs_dd(A, X0)
    return A, X0, D0, Xh, Xl, lam_t


def test_theorem1_bound():
    A, X0, D0, Xh, Xl, lam_t = _well_separated()
    n = A.shape[0]
    Xn, lam, info = rf.step(A, X0, D0, 1e-15, rf.Options())
    X1 = info["X1"]
    E = np.linalg.solve(X1, Xh + Xl) - np.eye(n)       # X = X^(1) (I + E), eq. E'
    eps = np.linalg.norm(E, 2)
    normA = np.max(np.abs(lam_t))
    gap = np.min(np.diff(np.sort(lam_t)))
    assert eps < min(gap / (10 * math.sqrt(n) * normA), 0.01)      # eq. assume1
    bound = 6.4 * math.sqrt(n) * normA * eps ** 2 / (gap - 14 * normA * eps)
    assert np.linalg.norm(E - info["E"], 2) <= bound


def test_quadratic_convergence():
    A, X0, D0, Xh, Xl, lam_t = _well_separated(rel=1e-4, seed=6)
    n = A.shape[0]
    normA = np.max(np.abs(lam_t))
    gap = np.min(np.diff(np.sort(lam_t)))
    hist = []
    rf.refine(A, X0, D0, 1e-15, rf.Options(max_iter=4), history=hist)
    fe = [tr.forward_error(Xh, Xl, X0)] + [tr.forward_error(Xh, Xl, h["X"]) for h in hist]
    assert fe[1] < 1e-6 and fe[2] < 1e-13
    for a, b in zip(fe[:-1], fe[1:]):
        assert b <= 6.4 * math.sqrt(n) * normA * a * a / (gap - 14 * normA * a) + 8 * U * math.sqrt(n)


def test_workload0_reaches_delta():
    A, X0, D0 = synth.workload0()
    Xh, Xl, _, _ = tr.eigvecs_dd(A, X0)
    X, lam, info = rf.refine(A, X0, D0, 1e-14, rf.Options())
    assert info["status"] == "converged" and info["iters"] <= 4
    assert tr.forward_error(Xh, Xl, X) <= 1e-14


@pytest.mark.parametrize("n,cond,pert,delta", [(64, 1e8, 1e-8, 1e-14), (48, 1e4, 1e-6, 1e-14),
                                                (64, 1e2, 1e-4, 1e-15)])
def test_stop_within_one_iteration_of_the_truth(n, cond, pert, delta):
    # the stopping estimate models the forward error after the step (the error model of
    # Sec. 3.2, quadratic in the step): with quadratic convergence the iteration stops no later
    # than one step after the true forward error first falls to delta, and never before it
    A, Q, lam = synth.symmetric_matrix(n, cond, 7, "spd")
    X0, D0 = synth.initial_guess(Q, lam, 7, pert)
    Xh, Xl, _, _ = tr.eigvecs_dd(A, X0)
    hist = []
    X, l, info = rf.refine(A, X0, D0, delta, rf.Options(), history=hist)
    assert info["status"] == "converged"
    fe = [tr.forward_error(Xh, Xl, h["X"]) for h in hist]
    first = next(k for k, e in enumerate(fe, 1) if e <= delta)
    assert first <= info["iters"] <= first + 1


def test_workload0_fixed_56_bit_a_floor():
    # 7 planes of A (56 bits) cannot resolve gaps of 3.4e-9 to 1e-14: the error stalls
    # near 2^-56 / gap and the iteration does not converge.
    A, X0, D0 = synth.workload0()
    Xh, Xl, _, _ = tr.eigvecs_dd(A, X0)
    X, lam, info = rf.refine(A, X0, D0, 1e-14, rf.Options(slices_A=7, max_iter=3))
    fe = tr.forward_error(Xh, Xl, X)
    assert info["status"] != "converged"
    assert 1e-10 < fe < 1e-8


def test_delta_must_exceed_u():
    A, X0, D0 = synth.workload0()
    with pytest.raises(ValueError):
        rf.refine(A, X0, D0, U, rf.Options())


def test_clusters_auto_rule_subspaces():
    n = 32
    A, Q, lam = synth.symmetric_matrix(n, 1e2, 5, "clustered", cluster_pairs=2, cluster_gap=1e-10)
    X0, D0 = synth.initial_guess(Q, lam, 5, 1e-8)
    Xh, Xl, _, _ = tr.eigvecs_dd(A, X0)
    X, l, info = rf.refine(A, X0, D0, 1e-12, rf.Options(cluster="auto"))
    assert info["status"] == "converged"
    ci = np.nonzero(np.diff(np.sort(lam)) < 1e-9)[0]
    assert len(ci) == 2
    mask = np.ones(n, bool)
    for i in ci:
        assert tr.subspace_error(Xh, Xl, X, [i, i + 1]) <= 1e-12
        mask[i] = mask[i + 1] = False
    assert tr.forward_error(Xh[:, mask], Xl[:, mask], X[:, mask]) <= 1e-12


def test_cluster_rule_restores_orthonormality_inside_a_cluster():
    # the true eigenvectors are orthonormal; a start whose clustered columns are mixed by a
    # non-orthogonal 2 x 2 (x_i^T x_j ~ 2e-6) is repaired by e~_ij = r_ij / 2 (R -> O(R^2) per
    # step) while the subspace stays put, so both the subspace and X^T X = I hold to delta
    n = 32
    A, Q, lam = synth.symmetric_matrix(n, 1e2, 5, "clustered", cluster_pairs=2, cluster_gap=1e-10)
    X0, D0 = synth.initial_guess(Q, lam, 5, 1e-8)
    ci = np.nonzero(np.diff(np.sort(lam)) < 1e-9)[0]
    for i in ci:
        X0[:, [i, i + 1]] = X0[:, [i, i + 1]] @ np.array([[1.0, 1e-6], [1e-6, 1.0]])
    Xh, Xl, _, _ = tr.eigvecs_dd(A, X0)
    X, l, info = rf.refine(A, X0, D0, 1e-12, rf.Options(cluster="auto"))
    assert info["status"] == "converged"
    G = X.T @ X - np.eye(n)
    for i in ci:
        J = [i, i + 1]
        assert np.abs(G[np.ix_(J, J)]).max() <= 1e-12
        assert tr.subspace_error(Xh, Xl, X, J) <= 1e-12


def test_truth_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    A, Q, lam = synth.symmetric_matrix(10, 1e3, 3)
    X0, _ = synth.initial_guess(Q, lam, 3, 1e-8)
    Xh, Xl, _, _ = tr.eigvecs_dd(A, X0)
    E, V = mpmath.eigsy(mpmath.matrix(A.tolist()))
    order = np.argsort([float(E[i]) for i in range(10)])
    Vh = np.array([[float(V[i, j]) for j in order] for i in range(10)])
    Vl = np.array([[float(V[i, j] - mpmath.mpf(float(V[i, j]))) for j in order] for i in range(10)])
    s = np.sign(np.sum(Vh * Xh, 0))
    assert np.max(np.abs((Xh - Vh * s) + (Xl - Vl * s))) <= 1e-28


def test_golden_workload0_regression():
    # tests/golden/workload0_oracle.json is written by tests/golden/make_golden.py (oracle only)
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "workload0_oracle.json")
    gold = json.load(open(path))
    A, X0, D0 = synth.workload0()
    Xh, Xl, _, _ = tr.eigvecs_dd(A, X0)
    hist = []
    _, _, info = rf.refine(A, X0, D0, 1e-14, rf.Options(), history=hist)
    assert info["status"] == gold["auto"]["status"] and info["iters"] == gold["auto"]["iters"]
    for h, gs in zip(hist, gold["auto"]["steps"]):
        for key in ("beta", "alpha", "sX", "kV", "kW", "kU", "products"):
            assert h[key] == gs[key]
        fe = tr.forward_error(Xh, Xl, h["X"])
        assert abs(fe - gs["forward_error"]) <= 1e-3 * gs["forward_error"] + 1e-16


def test_start_outside_the_basin_still_converges():
    # Exact-truth workload (Hadamard eigenvectors), n = 512, cond 1e12: gaps of 5.7e-14 put the
    # 1e-8 start far outside Theorem 1's basin.  The first correction raises the error (the
    # near-degenerate pairs mix), the second repairs it; one non-contracting step is not
    # stagnation, and the iteration reaches delta against the known eigenvectors.
    A, X0, D0, lam, Qh, Ql, info = synth.hadamard_workload(512, 1e12, synth.seed_for(4, 500))
    hist = []
    X, lam_out, res = rf.refine(A, X0, D0, 1e-14, rf.Options(), history=hist)

    def fe(Y):
        s = np.sign(np.sum(Qh * Y, 0))
        return np.linalg.norm((Y * s - Qh) - Ql, 2)

    assert fe(hist[0]["X"]) > 100 * fe(X0)          # the first step makes things worse
    assert hist[1]["step"] > 0.5 * hist[0]["step"]  # ... and the second step is as large
    assert res["status"] == "converged"
    assert fe(X) <= 1e-14


def test_previous_study_form_keeps_x_at_its_planes():
    # x_planes = 7 keeps X at 7 digit planes (56 bits on the column grid): every entry within
    # 2^(f-3) of the column maximum is unchanged, smaller ones are rounded to 2^(f-55)
    A, X0, D0 = synth.workload0()
    hist = []
    rf.refine(A, X0, D0, 1e-14, rf.Options(x_planes=7, max_iter=1), history=hist)
    p = rf.plan(A, X0, D0, 1e-14, rf.Options(x_planes=7))
    assert p["sX"] == 7 and p["beta"] == -2
    X1 = X0 - oz.slice_cols(X0, 7, p["f"])[2]
    big = np.abs(X0) >= np.ldexp(1.0, p["f"] - 3)[None, :]
    assert np.array_equal(X1[big], X0[big])
    assert np.all(np.abs(X1 - X0) <= np.ldexp(1.0, p["f"] - 56)[None, :])
    # three planes (24 bits): the tau grid of beta = 30
    p3 = rf.plan(A, X0, D0, 1e-14, rf.Options(x_planes=3))
    X13 = X0 - oz.slice_cols(X0, 3, p3["f"])[2]
    T, _ = oz.tau_truncate_cols(X0, 30, p3["f"])
    assert p3["sX"] == 3 and np.array_equal(X13, T)


def test_sparse_rule_is_the_paper_formula():
    # Sec. 4 (sparse matrices): beta = floor(log2(gamma min(k, sqrt n) / (0.75 u) sqrt(1 / S2))),
    # gamma = sqrt(delta gap / max|lam|), alpha = 53 - beta + ceil(log2 k), k = max row nonzeros
    n, bw, delta = 300, 2, 1e-12
    A, X0, D0, lam = synth.banded_workload(n, bw, 11)
    assert np.max(np.count_nonzero(A, axis=1)) == 2 * bw + 1
    p = rf.plan(A, X0, D0, delta, rf.Options(sparse_rule=True))
    k = 2 * bw + 1
    s = np.sort(D0)
    gap = np.min(np.diff(s))
    Lam = np.max(np.abs(D0))
    f = oz.col_exponents(X0)
    S2 = math.fsum(math.ldexp(1.0, 2 * int(e)) for e in f)
    gamma = math.sqrt(delta * gap / Lam)
    q = gamma * min(k, math.sqrt(n)) / (0.75 * U) * math.sqrt(1.0 / S2)
    beta = min(max(math.floor(math.log2(q)), 3), 47)
    assert p["beta"] == beta
    assert p["alpha"] == 53 - beta + 3
    # finer than the dense n delta form of Sec. 4.1: min(k, sqrt n)^2 = 25 < n keeps more bits of
    # X (smaller beta); coarser than xi = 1 (25 > 1)
    assert p["beta"] < rf.plan(A, X0, D0, delta, rf.Options(xi=None))["beta"]
    assert p["beta"] > rf.plan(A, X0, D0, delta, rf.Options(xi=1.0))["beta"]


def test_previous_study_step_works_on_x_at_its_planes():
    # the iteration itself (not only its plan) works on X kept at x_planes digit planes: with
    # three planes X^(1) is X rounded to the tau grid of beta = 30, exactly representable by
    # its three planes
    A, X0, D0 = synth.workload0()
    _, _, info = rf.step(A, X0, D0, 1e-14, rf.Options(x_planes=3))
    f = info["plan"]["f"]
    T, _ = oz.tau_truncate_cols(X0, 30, f)
    assert np.array_equal(info["X1"], T)
    assert not np.any(oz.slice_cols(info["X1"], 3, f)[2])


def test_sparse_rule_reduces_to_the_dense_form_when_k_is_sqrt_n():
    # Sec. 4 replaces sqrt n by min(k, sqrt n) in beta and ceil(log2 sqrt n) by ceil(log2 k) in
    # alpha.  A 64 x 64 matrix with exactly k = 8 = sqrt 64 nonzeros in every row (eight dense
    # symmetric 8 x 8 blocks) must get the beta and alpha of the dense n delta form of Sec. 4.1.
    g = np.random.default_rng(11)
    A = np.zeros((64, 64))
    for b in range(8):
        M = g.standard_normal((8, 8))
        A[8 * b:8 * b + 8, 8 * b:8 * b + 8] = M + M.T + 20.0 * np.eye(8) * (b + 1)
    assert np.all(np.count_nonzero(A, axis=1) == 8)
    lam, Q = np.linalg.eigh(A)
    X0 = Q + 1e-9 * g.standard_normal(Q.shape)
    for delta in (1e-10, 1e-13):
        ps = rf.plan(A, X0, lam, delta, rf.Options(sparse_rule=True))
        pd = rf.plan(A, X0, lam, delta, rf.Options(xi=None))
        assert ps["beta"] == pd["beta"] and ps["alpha"] == pd["alpha"]


def test_int32_plane_bound_is_the_largest_exact_count():
    # k anti-diagonal pairs of digit products (|d| <= 128, so |product| <= 2^14) summed over n
    # terms fit int32 exactly while k n 2^14 <= 2^31 - 1; int32_planes(n) is the largest such k
    for n in (1, 7, 64, 1000, 4096, 8192, 12288):
        k = rf.int32_planes(n)
        assert k * n * 128 * 128 <= 2 ** 31 - 1 < (k + 1) * n * 128 * 128


def _plan_case(lam_prev, omega_prev=0.0, col_max=0.25, xi=None):
    # n = 4, X = col_max * I: every column maximum is col_max, so f_j = ceil(log2 col_max);
    # A = I (only its exponents and nonzero counts enter the plan); the n delta form of Sec. 4.1
    # unless xi is given
    X = col_max * np.eye(4)
    return rf.plan(np.eye(4), X, np.asarray(lam_prev, dtype=np.float64), 2.0 ** -30, rf.Options(xi=xi),
                   omega_prev)


def test_plan_gap_and_beta_worked_by_hand():
    # Sec. 3.3 / Sec. 4.1 through the oracle's plan, with every input chosen so that the
    # result follows by hand:
    #   estimates (unsorted) 0.5, -1, 0.5 + 2^-20, 2  ->  sorted -1, 0.5, 0.5 + 2^-20, 2
    #   adjacent gaps 1.5, 2^-20, 1.5 - 2^-20  ->  smallest gap g = 2^-20;  max|lam| = 2
    #   columns of X = 0.25 I: f_j = -2, sum_j 2^(2 f_j) = 4 * 2^-4 = 1/4
    #   n delta g / (max|lam| S2) = 4 * 2^-30 * 2^-20 / (2 * 2^-2) = 2^-47;  sqrt = 2^-23.5
    #   2^-23.5 / (0.75 * 2^-53) = 2^29.5 * 4/3 = 2^29.915  ->  beta = floor = 29
    p = _plan_case([0.5, -1.0, 0.5 + 2.0 ** -20, 2.0])
    assert p["g"] == 2.0 ** -20 and p["Lam"] == 2.0
    assert p["f"].tolist() == [-2, -2, -2, -2] and p["S2"] == 0.25
    assert p["beta"] == 29
    # with xi = 1 in place of n = 4 the square root loses a factor 2: 2^28.915 -> beta = 28
    assert _plan_case([0.5, -1.0, 0.5 + 2.0 ** -20, 2.0], xi=1.0)["beta"] == 28
    # a gap at or below the cluster threshold omega = 2^-19 is not a gap: g = 1.5 - 2^-20;
    #   4 * 2^-30 * (1.5 - 2^-20) / (2 * 2^-2) = 2^-27 (1.5 - 2^-20); log2 of its square root
    #   = (0.58496 - 27) / 2 = -13.2075; + 53 + log2(4/3) = 40.2  ->  beta = 40
    p = _plan_case([0.5, -1.0, 0.5 + 2.0 ** -20, 2.0], omega_prev=2.0 ** -19)
    assert p["g"] == 1.5 - 2.0 ** -20 and p["beta"] == 40
    # a repeated estimate gives a zero gap, which is excluded too: g = 1.5
    p = _plan_case([0.5, -1.0, 0.5, 2.0])
    assert p["g"] == 1.5 and p["beta"] == 40
    # the largest magnitude is negative: max|lam| = 4 (not the largest value, 2);
    #   4 * 2^-50 / (4 * 2^-2) = 2^-48, sqrt 2^-24, / (0.75 * 2^-53) = 2^29.415 -> beta = 29
    p = _plan_case([0.5, -4.0, 0.5 + 2.0 ** -20, 2.0])
    assert p["Lam"] == 4.0 and p["g"] == 2.0 ** -20 and p["beta"] == 29
    # columns with maximum 2^-5 < 0.05 <= 2^-4: f_j = -4, S2 = 4 * 2^-8 = 2^-6, 16 times smaller:
    #   beta = floor(29.915 + log2 sqrt 16) = floor(31.915) = 31
    p = _plan_case([0.5, -1.0, 0.5 + 2.0 ** -20, 2.0], col_max=0.05)
    assert p["S2"] == 2.0 ** -6 and p["beta"] == 31
    # one estimate only: no gap exists and g = max|lam| (n = 1)
    g, Lam = rf.min_gap(np.array([-3.0]))
    assert g == 3.0 and Lam == 3.0


def test_sum_pow4_against_fractions():
    from fractions import Fraction
    cases = ([-1, -3, 0, 5, -40], [0] + [-30] * 3, [-1074 // 2 + 3, 10, 10, -7], list(range(-20, 21)),
             [oz.EZERO, -2, oz.EZERO, 3])
    for f in cases:
        exact = sum((Fraction(2) ** (2 * x) for x in f if x != oz.EZERO), Fraction(0))
        assert rf.sum_pow4(np.array(f)) == float(exact)      # correctly rounded
    assert rf.sum_pow4(np.array([3, 3])) == 128.0            # 2 * 2^6, not 2 * 2^3
    assert rf.sum_pow4(np.array([oz.EZERO])) == 0.0


def test_forward_error_closed_form():
    # X = I (exact), X^ = I + diag(3e-7, 0, -4e-7, 0, 1e-7, 0) with column 1 sign-flipped:
    # after the sign alignment of column 1 the difference is diagonal, so its 2-norm is the
    # largest |d_j| = 4e-7 (the Frobenius norm would be 5.1e-7; without the alignment, 2)
    n = 6
    d = np.array([3e-7, 0.0, -4e-7, 0.0, 1e-7, 0.0])
    Xhat = np.eye(n) + np.diag(d)
    Xhat[:, 1] *= -1.0
    fe = tr.forward_error(np.eye(n), np.zeros((n, n)), Xhat)
    # 1 - fl(1 + d_j) is exact (Sterbenz), so the diagonal differences are known exactly
    assert abs(fe - abs(1.0 - Xhat[2, 2])) <= 1e-9 * fe
    assert abs(fe - 4e-7) <= 1e-16
    # the low word of X counts: X = I + 2^-60 e_0 e_0^T held as (I, 2^-60 e_0 e_0^T), X^ = I
    Xl = np.zeros((n, n))
    Xl[0, 0] = 2.0 ** -60
    assert tr.forward_error(np.eye(n), Xl, np.eye(n)) == 2.0 ** -60


def test_forward_error_of_swapped_columns():
    # X = I, X^ = I with columns 0 and 1 swapped: x_i^T x^_i = 0 for both, so no sign can
    # bring them closer and each keeps its own sign.  The difference is zero outside the
    # leading 2 x 2 block [[1, -1], [-1, 1]], whose 2-norm is 2.
    n = 5
    Xhat = np.eye(n)[:, [1, 0, 2, 3, 4]]
    assert tr.forward_error(np.eye(n), np.zeros((n, n)), Xhat) == pytest.approx(2.0, rel=1e-15)


def test_forward_error_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    n = 7
    rng = np.random.default_rng(20260207)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Xl = rng.standard_normal((n, n)) * 1e-17 * np.abs(Q)
    Xhat = Q + rng.standard_normal((n, n)) * 1e-9
    flips = np.array([1, -1, 1, 1, -1, -1, 1], dtype=np.float64)
    fe = tr.forward_error(Q, Xl, Xhat * flips[None, :])
    D = mpmath.matrix(n, n)
    for i in range(n):
        for j in range(n):
            D[i, j] = mpmath.mpf(float(Q[i, j])) + mpmath.mpf(float(Xl[i, j])) - mpmath.mpf(float(Xhat[i, j]))
    s = mpmath.svd_r(D, compute_uv=False)
    ref = float(max(s[i] for i in range(n)))
    assert abs(fe - ref) <= 1e-6 * ref


def test_subspace_error_closed_form():
    # span(e0, e1) against the columns of X^ that tilt it by known principal angles:
    # x^_0 = 2 (cos a e0 + sin a e3), x^_1 = 0.5 (cos b e1 + sin b e4): the angles are a and b, so
    # ||sin Theta||_2 = max(sin a, sin b) whatever the columns' lengths (Frobenius would be
    # sqrt(sin^2 a + sin^2 b))
    n = 6
    I = np.eye(n)
    a, b = 0.3, 0.2
    Xhat = np.eye(n)
    Xhat[:, 0] = 2.0 * (np.cos(a) * I[:, 0] + np.sin(a) * I[:, 3])
    Xhat[:, 1] = 0.5 * (np.cos(b) * I[:, 1] + np.sin(b) * I[:, 4])
    se = tr.subspace_error(I, np.zeros((n, n)), Xhat, [0, 1])
    assert abs(se - np.sin(a)) <= 1e-15
    # a rotation and a scaling inside the subspace change no angle
    c, s = np.cos(0.7), np.sin(0.7)
    Xhat = np.eye(n)
    Xhat[:, 0] = 3.0 * (c * I[:, 0] + s * I[:, 1])
    Xhat[:, 1] = -s * I[:, 0] + c * I[:, 1]
    assert tr.subspace_error(I, np.zeros((n, n)), Xhat, [0, 1]) <= 1e-15


@pytest.mark.parametrize("seed", [1, 3])
def test_estimates_are_the_correctly_rounded_rayleigh_quotients(seed):
    # Alg. 1: lam_i = x_i^T v_i / (1 - r_i) with v_i = A x_i and 1 - r_i = x_i^T x_i,
    # the Rayleigh quotient of x_i = X^(1)[:, i].  With A's entries small integers, A lies
    # wholly in its first digit plane, so V holds A X^(1) to double-double accuracy, and the
    # estimate must be the quotient computed in exact rationals, rounded once.  beta = 2 keeps
    # X^(1) at 51 bits, so A X^(1) needs more than 53 and V's low words are nonzero.  An
    # indefinite A and columns unrelated to its eigenvectors make x^T A x cancel (up to several
    # hundred times smaller than |A x| |x|), which exposes a dropped low word of V or an FP64
    # division.
    from fractions import Fraction
    n = 40
    rng = np.random.default_rng(seed)
    B = rng.integers(-50, 51, size=(n, n)).astype(np.float64)
    A = np.triu(B) + np.triu(B, 1).T
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Xn, lam, info = rf.step(A, Q, np.linalg.eigvalsh(A), 1e-14, rf.Options(beta_override=2))
    assert info["sX"] <= info["kV"]                    # every pair with A's first plane is kept
    assert np.count_nonzero(info["Vl"]) > n * n // 2
    X1 = info["X1"]
    Af = [[Fraction(int(a)) for a in row] for row in A]
    for i in range(n):
        x = [Fraction(float(v)) for v in X1[:, i]]
        Ax = [sum(Af[r][c] * x[c] for c in range(n)) for r in range(n)]
        q = sum(x[r] * Ax[r] for r in range(n)) / sum(v * v for v in x)
        assert lam[i] == float(q), (i, lam[i], float(q))


@pytest.mark.parametrize("eps,clustered", [(2.0 ** -10, True), (2.0 ** -8, False)])
def test_auto_cluster_threshold_worked_by_hand(eps, clustered):
    # The automatic threshold omega = 2 (||W offdiag||_F + max|lam| ||r||_2) worked by hand on
    # A = diag(1, 1 + eps, 4) with X mixing the first two axes, x0 = (p, q, 0), x1 = (-q, p, 0),
    # x2 = e3, p = 1 - 2^-14, q = 2^-8 (beta = 2 keeps X^(1) = X).  With m = p^2 + q^2:
    #   lam0 = 1 + eps q^2 / m,  lam1 = 1 + eps p^2 / m,  lam2 = 4;  r0 = r1 = 1 - m, r2 = 0;
    #   w01 = w10 = eps p q (x0^T x1 = 0), every other off-diagonal w is 0;
    #   omega = 2 (sqrt 2 eps p q + 4 sqrt 2 (1 - m)) = 1.2192e-3 (eps = 2^-10), 1.2515e-3 (2^-8).
    # lam1 - lam0 = eps (p^2 - q^2) / m = 9.765e-4 lies below omega for eps = 2^-10 (a cluster
    # pair: e~01 = r01 / 2 = 0) but above omega / 2 and above 2 sqrt 2 (eps p q + 1 - m), and
    # 3.906e-3 lies above omega for eps = 2^-8 (e~01 = w01 / (lam1 - lam0) = p q m / (p^2 - q^2)).
    p, q = 1.0 - 2.0 ** -14, 2.0 ** -8
    m = p * p + q * q
    A = np.diag([1.0, 1.0 + eps, 4.0])
    X = np.array([[p, -q, 0.0], [q, p, 0.0], [0.0, 0.0, 1.0]])
    Xn, lam, info = rf.step(A, X, np.diag(A).copy(), 1e-14, rf.Options(cluster="auto", beta_override=2))
    assert np.array_equal(info["X1"], X)
    omega = 2.0 * math.sqrt(2.0) * (eps * p * q + 4.0 * (1.0 - m))
    assert info["omega"] == pytest.approx(omega, rel=1e-12)
    assert lam[1] - lam[0] == pytest.approx(eps * (p * p - q * q) / m, rel=1e-12)
    if clustered:
        assert info["E"][0, 1] == 0.0 and info["E"][1, 0] == 0.0
    else:
        e01 = p * q * m / (p * p - q * q)
        assert info["E"][0, 1] == pytest.approx(e01, rel=1e-12)
        assert info["E"][1, 0] == pytest.approx(-e01, rel=1e-12)


@pytest.mark.parametrize("k_cap,case", [(5, 0), (5, 1), (5, 2), (4, 0)])
def test_capped_products_stop_as_stagnated_at_their_floor(k_cap, case):
    # With every product capped at k_cap digit planes the iteration can only reach an error
    # floor far above delta (step norms about 4e-8 for 5 planes, 1e-5 for 4).  The stopping
    # rule for such a run (two consecutive steps that fail to halve) must end it as stagnated
    # within two iterations of the first step that fails to halve, with no step before that
    # one failing, rather than run on at the floor until max_iter.
    A, X0, D0, _ = synth.refine_workload(48, 1e4, case=case, rel=1e-6)
    hist = []
    X, lam, info = rf.refine(A, X0, D0, 1e-14, rf.Options(k_cap=k_cap, max_iter=12), history=hist)
    steps = [h["step"] for h in hist]
    first = next(i for i in range(1, len(steps)) if steps[i] > 0.5 * steps[i - 1])
    assert info["status"] == "stagnated"
    assert info["iters"] <= first + 2
    assert info["err_est"] > 50 * 1e-14                     # the floor lies far above delta
    assert min(steps[first:]) > 0.1 * steps[first]         # the run hovers at its floor


def test_beta_clamped_so_x1_keeps_its_leading_bits():
    # A loose target asks for a coarse truncation: on this 2 x 2 problem at delta = 0.01 the
    # Sec. 4.1 rule gives floor(log2 q) = 49.  beta is clamped to 47, so X^(1) lies on the grid
    # ulp(tau_j) = 2^(f_j + beta - 53) = 2^(f_j - 6) and keeps its leading 7 bits (one digit
    # plane); near beta = 53 that grid reaches 2^f_j and X^(1) would keep no bits at all.
    A = np.array([[2.0, 0.5], [0.5, 1.0]])
    w, Q = np.linalg.eigh(A)
    X = Q + 1e-3 * np.array([[0.3, -0.2], [0.1, 0.4]])
    p = rf.plan(A, X, w, 0.01, rf.Options())
    assert p["f"].tolist() == [0, 0] and p["beta"] == 47 and p["sX"] == 1
    g, Lam = rf.min_gap(w)
    q = math.sqrt(0.01 * g / (Lam * rf.sum_pow4(p["f"]))) / (0.75 * U)
    assert math.floor(math.log2(q)) == 49
    Xn, lam, info = rf.step(A, X, w, 0.01, rf.Options())
    grid = 2.0 ** -6
    assert np.array_equal(info["X1"], np.round(X / grid) * grid)   # np.round: ties to even
    assert np.all(info["X1"] != 0.0)


def test_v_slices_cover_the_largest_column():
    # The slice count of V = A X^(1) bounds the dropped part by tau = delta gap for every
    # column at once, so it is set by the largest column exponent.  With one column scaled
    # down by 2^-24 the exponents span 24 bits (three planes), and the dropped part measured
    # against A X^(1) formed in double-double must still stay below tau in the 2-norm.
    A, X0, D0, _ = synth.refine_workload(48, 1e4, case=0, rel=1e-6)
    X = X0.copy()
    X[:, 0] *= 2.0 ** -24
    delta = 1e-12
    Xn, lam, info = rf.step(A, X, D0, delta, rf.Options())
    f = info["plan"]["f"]
    assert int(np.max(f)) - int(np.min(f)) >= 24
    Vh, Vl = dd.dd_matmul(A, None, info["X1"], None)
    err = np.linalg.norm((info["Vh"] - Vh) + (info["Vl"] - Vl), 2)
    assert err <= delta * info["plan"]["g"]


@pytest.mark.parametrize("case", [0, 1])
def test_each_product_within_its_tau(case):
    # The slice rule sets each product's planes so that what it drops stays below its own tau
    # in the 2-norm: delta * gap for V = A X^(1) and W = X^(1)^T Res, delta for the update
    # product U = X^(1) E~.  Each is measured here against the same product formed in
    # double-double from the step's own operands.
    A, X0, D0, _ = synth.refine_workload(64, 1e8, case=case, rel=1e-8)
    delta = 1e-14
    Xn, lam, info = rf.step(A, X0, D0, delta, rf.Options())
    X1, g = info["X1"], info["plan"]["g"]
    Vh, Vl = dd.dd_matmul(A, None, X1, None)
    assert np.linalg.norm((info["Vh"] - Vh) + (info["Vl"] - Vl), 2) <= delta * g
    Wh, Wl = dd.dd_matmul(X1.T, None, info["Res"], None)
    assert np.linalg.norm((info["W"] - Wh) - Wl, 2) <= delta * g
    Uh, Ul = dd.dd_matmul(X1, None, info["E"], None)
    assert np.linalg.norm((info["Uh"] - Uh) + (info["Ul"] - Ul), 2) <= delta


def test_residual_is_the_correctly_rounded_difference():
    # Res = V - X^(1) diag(lam) formed in double-double and rounded once (Alg. 1's residual):
    # on sampled entries it equals the exact rational value of Vh + Vl - x1_ij lam_j rounded to
    # nearest.  The entries cancel by about eight digits here (V ~ X^(1) diag(lam)), so a low
    # word dropped on either side shows.
    from fractions import Fraction as Fr
    A, X0, D0 = synth.workload0()
    Xn, lam, info = rf.step(A, X0, D0, 1e-14, rf.Options())
    X1, Vh, Vl, Res = info["X1"], info["Vh"], info["Vl"], info["Res"]
    g = np.random.default_rng(11)
    for i, j in zip(g.integers(0, 64, 400), g.integers(0, 64, 400)):
        ex = Fr(Vh[i, j]) + Fr(Vl[i, j]) - Fr(X1[i, j]) * Fr(lam[j])
        assert Res[i, j] == float(ex), (i, j)
