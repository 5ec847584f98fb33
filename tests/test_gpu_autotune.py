"""The tile autotuner of the slice products: every tile configuration gives the same bits, and
the tuner decides by timing, by its cost model, or from its cache as documented in frx.h.

Every tile sum of a slice product is an exact integer, so the tile configuration (128 x 128 or
128 x 256 tiles per CTA) can change the time of a product but never its result: ozaki_gemm, refine and refine_batched must
return identical bits under every forced configuration and under the tuner's own choice.  The
oracle pins their common result on a ragged ozaki_gemm."""
import numpy as np
import pytest

from oracle import ozaki as oz
from paper_2602_19090_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2602_19090_gb300 import api as a
    yield a
    a.set_tile("auto")


def G():
    from tests import gpu_util
    return gpu_util


def _forced(api, w, fn):
    prev = api.set_tile(w)
    try:
        return fn()
    finally:
        api.set_tile(prev)


CFGS = ("128x128", "128x256")


@pytest.mark.parametrize("m,K,n,k,mode", [(300, 257, 190, 6, "full"), (129, 1000, 385, 8, "triangular"),
                                          (1024, 1024, 1024, 8, "triangular"), (640, 4096, 1000, 4, "full")])
def test_ozaki_gemm_same_bits_in_every_tile_configuration(api, m, K, n, k, mode):
    # ragged rows (300, 129: a last tile row mostly past the end), ragged columns and a long
    # inner dimension
    g = G()
    A = synth.gemm_operand(m, K, 2.0, 700 + m)
    B = synth.gemm_operand(K, n, 2.0, 701 + n)
    Ad, Bd = g.to_dev(A), g.to_dev(B)
    out = {}
    for w in CFGS + ("auto",):
        Ch, Cl = _forced(api, w, lambda: api.ozaki_gemm(Ad, Bd, k, mode, return_lo=True))
        if w != "auto":
            assert api.last_tile() == w
        out[w] = (Ch.cpu().numpy(), Cl.cpu().numpy())
    for w in ("128x256", "auto"):
        assert np.array_equal(out[w][0], out["128x128"][0]) and np.array_equal(out[w][1], out["128x128"][1])
    if m * n * K <= 40_000_000:
        C_ref, o = oz.ozaki_gemm(A, B, k, mode)
        mag = np.abs(A) @ np.abs(B)
        hi, lo = out["128x128"]
        assert np.all(np.abs((hi - o["hi"]) + (lo - o["lo"])) <= mag * 2.0 ** -100)


def test_refine_same_bits_in_every_tile_configuration(api):
    g = G()
    A, X0, D0, _ = synth.refine_workload(300, 1e6, "indefinite", case=31)
    res = {}
    for w in CFGS:
        X, D = g.to_dev(X0), g.to_dev(D0)
        info = _forced(api, w, lambda: api.refine(g.to_dev(A), X, D, 1e-14, api.Options(cluster_omega=-1.0)))
        assert api.last_tile() == w
        res[w] = (X.cpu().numpy(), D.cpu().numpy(), info)
    for w in CFGS[1:]:
        assert np.array_equal(res[w][0], res[CFGS[0]][0]) and np.array_equal(res[w][1], res[CFGS[0]][1])
        # the norms behind the stopping test are summed per column in a fixed order, so the
        # estimate repeats bit for bit as well
        for key in ("status", "iters", "products", "err_est", "step", "omega", "min_gap"):
            assert res[w][2][key] == res[CFGS[0]][2][key]


def test_refine_batched_same_bits_at_both_widths_and_tuned(api):
    g = G()
    sizes, conds = synth.batched_sizes(12, 32, 512, case=5)
    probs = [synth.refine_workload(int(nn), float(c), "spd", case=900 + b) for b, (nn, c) in
             enumerate(zip(sizes, conds))]
    res = {}
    for w in ("128x128", "128x256", "auto"):
        Xs = [g.to_dev(p[1]) for p in probs]
        Ds = [g.to_dev(p[2]) for p in probs]
        infos = _forced(api, w, lambda: api.refine_batched([g.to_dev(p[0]) for p in probs], Xs, Ds, 1e-12))
        if w != "auto":
            assert api.last_tile() == w
        res[w] = ([x.cpu().numpy() for x in Xs], [d.cpu().numpy() for d in Ds], infos)
    for w in ("128x256", "auto"):
        for b in range(len(probs)):
            assert np.array_equal(res[w][0][b], res["128x128"][0][b])
            assert np.array_equal(res[w][1][b], res["128x128"][1][b])
            assert res[w][2][b]["iters"] == res["128x128"][2][b]["iters"]


def test_tuner_times_ragged_products_and_caches_them(api):
    # a small ragged product is timed once; the same shape again is a cache hit; a large
    # square product whose wide tiles cover it exactly is settled by the cost model
    g = G()
    api.set_tile("auto")
    api.tune_stats(clear=True)
    A = g.to_dev(synth.gemm_operand(200, 300, 1.0, 720))
    B = g.to_dev(synth.gemm_operand(300, 170, 1.0, 721))
    api.ozaki_gemm(A, B, 4, "full")
    st = api.tune_stats()
    assert st["measured"] == 1 and st["modelled"] == 0
    first = api.last_tile()
    api.ozaki_gemm(A, B, 4, "full")
    st = api.tune_stats()
    assert st["measured"] == 1 and st["hits"] >= 1 and api.last_tile() == first
    n = 4096
    A = g.to_dev(synth.gemm_operand(n, n, 1.0, 722))
    B = g.to_dev(synth.gemm_operand(n, n, 1.0, 723))
    api.ozaki_gemm(A, B, 2, "full")
    st = api.tune_stats()
    assert st["measured"] == 1 and st["modelled"] == 1 and api.last_tile() == "128x256"


def test_set_tile_rejects_other_values(api):
    from paper_2602_19090_gb300.api import FrxError
    with pytest.raises(FrxError):
        api.set_tile(3)
    with pytest.raises(FrxError):
        api.set_tile(7)
    assert api.set_tile("auto") in CFGS + ("auto",)
