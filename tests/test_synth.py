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
