"""Parity at the benchmark's full sizes, in the launch configurations bench.py times.

* one refinement step of the n = 4096 workload (SPD, geometric spectrum cond 1e4, start
  perturbed by 1e-8, delta = 1e-14), every output of the step against the oracle;
* the Ozaki GEMM at n = 4096 (8 planes, both product sets, phi = 2), every entry;
* the Ozaki GEMM at n = 8192 on 256 seeded rows and columns (row and column exponents are
  per row and per column, so a block of the product is sliced exactly as in the full one);
* one refinement step at n = 11776, where the residual runs in 128-thread blocks, checked by
  size-independent properties against FP64 computations of the same quantities.
"""
import numpy as np
import pytest

from oracle import ozaki as oz
from oracle import refine as orf
from paper_2602_19090_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2602_19090_gb300 import api as a
    return a


def G():
    from tests import gpu_util
    return gpu_util


def test_refine_step_n4096_all_outputs(api):
    from tests.test_gpu_parity import _step_compare
    A, X0, D0, lam = synth.refine_workload(4096, 1e4, "spd", case=0)
    info, oi = _step_compare(api, A, X0, D0, 1e-14, orf.Options(), api.Options())
    assert info["k_V"] == 11 and info["s_X"] == 5     # the plan of the timed workload


def _gemm_compare(Ch, Cl, A, B, k, mode):
    C_ref, o = oz.ozaki_gemm(A, B, k, mode)
    mag = np.abs(A) @ np.abs(B)
    assert np.all(np.abs((Ch - o["hi"]) + (Cl - o["lo"])) <= mag * 2.0 ** -100)
    assert np.all(np.abs(Ch - C_ref) <= np.spacing(np.abs(C_ref)))
    assert np.mean(Ch == C_ref) > 0.999


@pytest.mark.parametrize("mode", ["triangular", "full"])
def test_ozaki_gemm_n4096_every_entry(api, mode):
    g = G()
    n, k = 4096, 8
    A = synth.gemm_operand(n, n, 2.0, synth.seed_for(1, 0))
    B = synth.gemm_operand(n, n, 2.0, synth.seed_for(1, 1))
    Ch, Cl = api.ozaki_gemm(g.to_dev(A), g.to_dev(B), k, mode, return_lo=True)
    _gemm_compare(Ch.cpu().numpy(), Cl.cpu().numpy(), A, B, k, mode)


def test_ozaki_gemm_n8192_sampled_block(api):
    g = G()
    n, k = 8192, 6
    A = synth.gemm_operand(n, n, 4.0, synth.seed_for(1, 2))
    B = synth.gemm_operand(n, n, 4.0, synth.seed_for(1, 3))
    Ch, Cl = api.ozaki_gemm(g.to_dev(A), g.to_dev(B), k, "triangular", return_lo=True)
    rng = synth.rng(synth.seed_for(1, 4))
    I = np.sort(rng.choice(n, 256, replace=False))
    J = np.sort(rng.choice(n, 256, replace=False))
    I[-1], J[-1] = n - 1, n - 1                       # the last row and column tile
    Ch = Ch.cpu().numpy()[np.ix_(I, J)]
    Cl = Cl.cpu().numpy()[np.ix_(I, J)]
    _gemm_compare(Ch, Cl, A[I, :], B[:, J], k, "triangular")


def test_refine_step_with_narrow_residual_blocks(api):
    # n = 11776 (> 11648): the residual's V column and the copy stages of 256-thread blocks would
    # pass 220 KB of shared memory, so it runs in 128-thread blocks, a configuration no smaller
    # case reaches.  A block-diagonal A with known eigenpairs: 184 blocks V_b diag(w_b) V_b^T,
    # V_b random orthogonal, w_b = 2 b + linspace(1, 2, 64) (gaps >= 1/63 inside a block, 1
    # between blocks, max |lambda| about 370).  After one step from a start perturbed by 1e-8,
    # checked by properties that hold at any size against FP64 computations of the same
    # quantities (tolerances above their own rounding errors, about 64 u max|lambda|): the
    # estimates are the Rayleigh quotients of X^(1) and match the spectrum, Res is the residual
    # they define, and X is orthonormal far beyond the start.
    import torch
    n, bs = 11776, 64
    rng = np.random.default_rng(synth.seed_for(5, n))
    A = np.zeros((n, n))
    Q = np.zeros((n, n))
    lam = np.empty(n)
    for b in range(n // bs):
        V, _ = np.linalg.qr(rng.standard_normal((bs, bs)))
        w = 2.0 * b + np.linspace(1.0, 2.0, bs)
        sl = slice(b * bs, (b + 1) * bs)
        A[sl, sl] = (V * w[None, :]) @ V.T
        A[sl, sl] = 0.5 * (A[sl, sl] + A[sl, sl].T)
        Q[sl, sl] = V
        lam[sl] = w
    X0 = Q + 1e-8 * rng.standard_normal((n, n)) * (Q != 0)
    dev = torch.device("cuda", 0)
    At = torch.from_numpy(A).to(dev)
    Xt = torch.from_numpy(X0).to(dev)
    Dt = torch.from_numpy(lam.copy()).to(dev)
    G0 = Xt.T @ Xt
    G0.diagonal().sub_(1.0)
    g0 = float(G0.abs().max())
    del G0
    info, mats = api.refine_step(At, Xt, Dt, 1e-12, api.Options())
    assert info["status"] >= 0
    Lam = float(np.max(np.abs(lam)))
    tol = 1e-13 * Lam
    assert np.max(np.abs(Dt.cpu().numpy() - lam)) <= 1e-12 * Lam
    X1 = mats["X1"]
    for b in range(0, n // bs, 23):
        sl = slice(b * bs, (b + 1) * bs)
        Xb, Ab = X1[sl, sl], At[sl, sl]
        rq = torch.diag(Xb.T @ Ab @ Xb) / torch.diag(Xb.T @ Xb)
        assert float((rq - Dt[sl]).abs().max()) <= tol
    R_ref = At @ X1 - X1 * Dt[None, :]
    assert float((mats["Res"] - R_ref).abs().max()) <= tol
    assert float(R_ref.abs().max()) > 100.0 * tol         # the residual is far from negligible
    del R_ref
    G = Xt.T @ Xt
    G.diagonal().sub_(1.0)
    g1 = float(G.abs().max())
    assert g1 <= 1e-7 and g1 <= 0.1 * g0
