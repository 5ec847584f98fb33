"""Parity at the benchmark's full sizes, in the launch configurations bench.py times.

* one refinement step of the n = 4096 workload (SPD, geometric spectrum cond 1e4, start
  perturbed by 1e-8, delta = 1e-14), every output of the step against the oracle;
* the Ozaki GEMM at n = 4096 (8 planes, both product sets, phi = 2), every entry;
* the Ozaki GEMM at n = 8192 on 256 seeded rows and columns (row and column exponents are
  per row and per column, so a block of the product is sliced exactly as in the full one).
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
