"""Measured forward error of frx_refine against known eigenvectors (the paper's target quantity).

* Exact-truth matrices (rotated Hadamard eigenvectors, not FP64 numbers, geometric spectrum)
  at n = 2048, cond 1e4 and 1e10, delta = 1e-14: ||X - X^||_2 <= delta, with the iteration
  and product counts of the CPU oracle on the same inputs.
* The reference X that bench.py uses for randsvd-like matrices (the native-FP64 comparator in
  its Sec. 4.1 form, iterated to delta = 1e-16) agrees with the oracle's double-double
  eigenvectors.
"""
import numpy as np
import pytest

from oracle import refine as orf
from oracle import truth as tr
from paper_2602_19090_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_19090_gb300 import api as a
    return a


def G():
    from tests import gpu_util
    return gpu_util


@pytest.mark.parametrize("cond", [1e4, 1e10])
def test_refine_n2048_exact_truth_within_delta(api, cond):
    g = G()
    n, delta = 2048, 1e-14
    A, X0, D0, lam, Qh, Ql, info = synth.rotated_hadamard_workload(n, cond, synth.seed_for(2, 900))
    X = g.to_dev(X0)
    res = api.refine(g.to_dev(A), X, g.to_dev(D0), delta)
    Xg = X.cpu().numpy()
    fe = tr.forward_error(Qh, Ql, Xg)
    assert res["status"] == 0
    assert fe <= delta
    assert tr.forward_error(Qh, Ql, X0) > 1e-9          # the start was 1e-8 away
    Xo, lo, oi = orf.refine(A, X0, D0, delta, orf.Options())
    assert oi["status"] == "converged"
    assert res["iters"] == oi["iters"] and res["products"] == oi["products"]
    assert tr.forward_error(Qh, Ql, Xo) <= delta


def test_fp64_reference_matches_the_oracle_truth(api):
    import torch

    from paper_2602_19090_gb300 import fp64_refine
    n = 200
    A, X0, D0, lam = synth.refine_workload(n, 1e10, "spd", case=600 + n % 97)
    Xh, Xl, _, _ = tr.eigvecs_dd(A, X0)
    dev = torch.device("cuda", 0)
    T, _, it = fp64_refine.refine(torch.from_numpy(A).to(dev), torch.from_numpy(X0).to(dev),
                                  torch.from_numpy(D0).to(dev), 1e-16, max_iter=8, xi=0.0)
    assert it["status"] == "converged"
    assert tr.forward_error(Xh, Xl, T.cpu().numpy()) <= 1e-15
