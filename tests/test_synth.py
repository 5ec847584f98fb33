"""The seeded input generators keep the promises the measurements rely on (CPU only).

The exact-truth workload's eigenvectors are known exactly; the randsvd-like matrices are exactly
symmetric with the geometric spectrum asked for; the generators are deterministic per seed.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2602_19090_gb300 import synth


@pytest.mark.parametrize("n,variant", [(64, "spd"), (128, "indefinite"), (256, "spd")])
def test_hadamard_workload_eigenpairs_are_exact(n, variant):
    A, X0, D0, lam, Qh, Ql, info = synth.hadamard_workload(n, 1e10, synth.seed_for(4, n), variant=variant)
    assert np.array_equal(A, A.T)
    # A = H diag(lam) H / n exactly: scaled by 2^S n, A is an integer matrix whose product with
    # H (entries +-1) is H diag(lam 2^S) n, checked in exact integer arithmetic
    S = -info["scale_exp"]
    Ai = A * (2.0 ** S * n)
    assert np.array_equal(Ai, np.rint(Ai))
    Ai = Ai.astype(np.int64).astype(object)
    H = np.sign(Qh).astype(np.int64).astype(object)       # columns ordered like lam
    lam_i = lam * 2.0 ** S
    assert np.array_equal(lam_i, np.rint(lam_i))
    lam_i = lam_i.astype(np.int64).astype(object)
    assert np.array_equal(Ai.dot(H), H * (lam_i * n)[None, :])
    # Q = Qh + Ql = H / sqrt(n) to double-double accuracy: (Qh + Ql)^2 n = 1 within 2^-100
    for v in (Fraction(float(Qh[0, 0])) + Fraction(float(Ql[0, 0])),
              Fraction(float(Qh[-1, -1])) + Fraction(float(Ql[-1, -1]))):
        assert abs(v * v * n - 1) < Fraction(1, 2 ** 100)
    assert np.all(np.diff(lam) > 0) and info["min_gap"] == float(np.min(np.diff(lam)))
    if variant == "spd":
        assert np.all(lam > 0)


@pytest.mark.parametrize("n,variant", [(8, "spd"), (64, "indefinite"), (128, "spd")])
def test_rotated_hadamard_workload_eigenpairs_are_exact(n, variant):
    A, X0, D0, lam, Qh, Ql, info = synth.rotated_hadamard_workload(n, 1e10, synth.seed_for(4, n), variant=variant)
    assert np.array_equal(A, A.T)
    # scaled by 2^S n, A is an integer matrix; Q 5 sqrt(n) = H R5 has entries +-7, +-1 and
    # A (H R5) = (H R5) diag(lam) is checked in exact integer arithmetic (times 2^S n)
    S = -info["scale_exp"]
    Ai = A * (2.0 ** S * n)
    assert np.array_equal(Ai, np.rint(Ai))
    Ai = Ai.astype(np.int64).astype(object)
    G = np.rint(Qh / np.abs(Qh).min()).astype(np.int64)      # H R5 (entries +-7, +-1)
    assert set(np.unique(np.abs(G)).tolist()) == {1, 7}
    # columns of H R5 are orthogonal with squared norm 25 n (so Q = H R5 / (5 sqrt n))
    Go = G.astype(object)
    assert np.array_equal(Go.T.dot(Go), np.eye(n, dtype=np.int64).astype(object) * (25 * n))
    lam_i = lam * 2.0 ** S
    assert np.array_equal(lam_i, np.rint(lam_i))
    lam_i = lam_i.astype(np.int64).astype(object)
    assert np.array_equal(Ai.dot(Go), Go * (lam_i * n)[None, :])
    # Qh + Ql = G / (5 sqrt n) to double-double accuracy
    for i, j in ((0, 0), (n - 1, n - 1), (1, n // 2)):
        v = Fraction(float(Qh[i, j])) + Fraction(float(Ql[i, j]))
        assert abs(v * v * 25 * n - G[i, j] ** 2) < Fraction(int(G[i, j]) ** 2, 2 ** 100)
    assert np.all(np.diff(lam) > 0) and info["min_gap"] == float(np.min(np.diff(lam)))
    if variant == "spd":
        assert np.all(lam > 0)
    assert abs(info["cond"] / 1e10 - 1) < 0.01


def test_randsvd_like_matrix_is_symmetric_with_the_geometric_spectrum():
    n, cond = 96, 1e6
    A, Q, lam = synth.symmetric_matrix(n, cond, synth.seed_for(2, 9))
    assert np.array_equal(A, A.T)
    assert np.allclose(Q.T @ Q, np.eye(n), atol=1e-14)
    ls = np.sort(lam)
    assert np.isclose(ls[-1] / ls[0], cond, rtol=1e-12)
    ratios = ls[1:] / ls[:-1]
    assert np.allclose(ratios, ratios[0], rtol=1e-12)              # geometric
    # the stored A is Q diag(lam) Q^T up to its own rounding
    assert np.abs(A - (Q * lam) @ Q.T).max() <= 64 * 2.0 ** -53 * ls[-1]


def test_generators_are_deterministic_per_seed():
    a = synth.refine_workload(40, 1e3, "indefinite", case=3)
    b = synth.refine_workload(40, 1e3, "indefinite", case=3)
    c = synth.refine_workload(40, 1e3, "indefinite", case=4)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert not np.array_equal(a[0], c[0])
    s1, c1 = synth.batched_sizes(64, case=1)
    s2, c2 = synth.batched_sizes(64, case=1)
    assert np.array_equal(s1, s2) and np.array_equal(c1, c2)
    assert s1.min() >= 32 and s1.max() <= 512


def test_random_sparse_workload_is_symmetric_sparse_and_seeded():
    A, X0, D0, lam = synth.random_sparse_workload(200, 8, 5)
    assert np.array_equal(A, A.T)
    nnz = np.count_nonzero(A, axis=1)
    assert nnz.min() >= 5 and nnz.max() <= 20
    assert np.allclose(X0.T @ X0, np.eye(200), atol=1e-13)
    B = synth.random_sparse_workload(200, 8, 5)[0]
    assert np.array_equal(A, B)
