"""Parity of the CUDA path with the CPU oracle (run on a GB300: pytest -m gpu)."""

import numpy as np
import pytest

from oracle import ozaki as oz
from oracle import refine as orf
from oracle import truth as tr
from paper_2602_19090_gb300 import synth

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def api():
    from paper_2602_19090_gb300 import api as a
    return a


def G():
    from tests import gpu_util
    return gpu_util


@pytest.mark.parametrize("phi", [0.5, 2.0, 4.0])
def test_exponents_bit_exact(api, phi):
    g = G()
    M = synth.gemm_operand(201, 133, phi, 100)
    M[7, :] = 0.0
    M[:, 5] = 0.0
    M[3, 3] = 2.0 ** -1060          # subnormal entry in a row with other entries
    Mt = g.to_dev(M)
    e0 = api.exponents(Mt, 0).cpu().numpy()
    e1 = api.exponents(Mt, 1).cpu().numpy()
    assert np.array_equal(e0, oz.row_exponents(M))
    assert np.array_equal(e1, oz.col_exponents(M))


def test_exponents_reject_nonfinite(api):
    g = G()
    M = np.ones((40, 30))
    M[4, 9] = np.nan
    with pytest.raises(api.FrxError) as ex:
        api.exponents(g.to_dev(M), 1)
    assert ex.value.status == -2


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("phi", [0.5, 4.0])
def test_slice_planes_bit_exact(api, axis, phi):
    g = G()
    M = synth.gemm_operand(150, 97, phi, 101 + axis)
    M[11, :] = 0.0
    Mt = g.to_dev(M)
    e = api.exponents(Mt, axis)
    k = 9
    planes = api.slice_planes(Mt, axis, e, k)
    d = g.bf16_digits(planes)
    if axis == 0:
        ref, _, _ = oz.slice_rows(M, k)                 # (k, rows, cols)
    else:
        ref, _, _ = oz.slice_cols(M, k)                 # (k, rows, cols) -> lines = cols
        ref = np.transpose(ref, (0, 2, 1))
    lines, other = ref.shape[1], ref.shape[2]
    assert np.array_equal(d[:, :lines, :other], ref)
    assert np.all(d[:, :, other:] == 0)


@pytest.mark.parametrize("m,n,K,kL,kR,T", [(200, 150, 300, 4, 3, 5), (64, 64, 64, 8, 6, 9),
                                           (130, 70, 1000, 3, 3, 6), (1, 1, 1, 2, 2, 4)])
def test_plane_products_bit_exact(api, m, n, K, kL, kR, T):
    g = G()
    L = synth.gemm_operand(m, K, 2.0, 200)
    R = synth.gemm_operand(K, n, 2.0, 201)
    Lt, Rt = g.to_dev(L), g.to_dev(R)
    eL = api.exponents(Lt, 0)
    eR = api.exponents(Rt, 1)
    Lp = api.slice_planes(Lt, 0, eL, kL)
    Rp = api.slice_planes(Rt, 1, eR, kR)
    out, gs = api.plane_products(Lp, Rp, K, kL, kR, T)
    dL, _, _ = oz.slice_rows(L, kL)
    dR, _, _ = oz.slice_cols(R, kR)
    S = oz.slice_products(dL, dR, oz.pair_set(kL, kR, T))
    ref = g.group_sums(S, kL, kR, T, gs)
    got = out.cpu().numpy()
    for gi, Rg in enumerate(ref):
        assert np.array_equal(got[gi].T.astype(object), Rg)


def test_plane_products_worst_case_digits(api):
    # all digits +128 (the largest 8-bit digit): every partial sum is as large as the
    # exactness bound allows
    g = G()
    K, kL, kR = 2048, 4, 4
    M = np.ones((64, K))
    Lt = g.to_dev(M)
    eL = api.exponents(Lt, 0)
    Lp = api.slice_planes(Lt, 0, eL, kL)
    d = g.bf16_digits(Lp)
    assert np.all(d[0, :, :K] == 128)
    Rp = Lp.clone()
    out, gs = api.plane_products(Lp, Rp, K, kL, kR, 2 * max(kL, kR))
    dL = d[:, :, :K]
    S = oz.slice_products(dL, np.transpose(dL, (0, 2, 1)), oz.pair_set(kL, kR, 8))
    ref = g.group_sums(S, kL, kR, 8, gs)
    for gi, Rg in enumerate(ref):
        assert np.array_equal(out.cpu().numpy()[gi].T.astype(object), Rg)


@pytest.mark.parametrize("mode", ["full", "triangular"])
@pytest.mark.parametrize("phi", [0.5, 2.0, 4.0])
def test_ozaki_gemm_matches_oracle(api, mode, phi):
    g = G()
    m, K, n, k = 150, 190, 70, 6
    A = synth.gemm_operand(m, K, phi, 300)
    B = synth.gemm_operand(K, n, phi, 301)
    Ch, Cl = api.ozaki_gemm(g.to_dev(A), g.to_dev(B), k, mode, return_lo=True)
    C_ref, o = oz.ozaki_gemm(A, B, k, mode)
    Ch = Ch.cpu().numpy()
    Cl = Cl.cpu().numpy()
    mag = np.abs(A) @ np.abs(B)
    assert np.all(np.abs((Ch - o["hi"]) + (Cl - o["lo"])) <= mag * 2.0 ** -100)
    assert np.all(np.abs(Ch - C_ref) <= np.spacing(np.abs(C_ref)))
    assert np.mean(Ch == C_ref) > 0.999


def test_ozaki_gemm_exact_inputs_correctly_rounded(api):
    g = G()
    A = synth.gemm_operand(40, 33, 0.5, 310)
    B = synth.gemm_operand(33, 20, 0.5, 311)
    C = api.ozaki_gemm(g.to_dev(A), g.to_dev(B), 12, "full").cpu().numpy()
    C_ref, _ = oz.ozaki_gemm(A, B, 12, "full", exact=True)
    assert np.array_equal(C, C_ref)


def _step_compare(api, A, X0, D0, delta, opts_o, opts_g):
    g = G()
    At, Xt, Dt = g.to_dev(A), g.to_dev(X0), g.to_dev(D0)
    info, mats = api.refine_step(At, Xt, Dt, delta, opts_g)
    Xn, lam, oi = orf.step(A, X0, D0, delta, opts_o)
    for key in ("beta", "alpha", "sX", "kV", "kW", "kU"):
        gk = {"sX": "s_X", "kV": "k_V", "kW": "k_W", "kU": "k_U"}.get(key, key)
        assert info[gk] == oi[key], key
    X1 = mats["X1"].cpu().numpy()
    assert np.array_equal(X1, oi["X1"])
    Vh, Vl = mats["Vh"].cpu().numpy(), mats["Vl"].cpu().numpy()
    vmag = np.abs(A) @ np.abs(X1)
    assert np.all(np.abs((Vh - oi["Vh"]) + (Vl - oi["Vl"])) <= vmag * 2.0 ** -100)
    assert np.allclose(mats["r"].cpu().numpy(), oi["r"], rtol=0, atol=4 * U * 1e-6)
    lam_g = Dt.cpu().numpy()
    assert np.all(np.abs(lam_g - lam) <= 2 * np.spacing(np.abs(lam)))
    Res = mats["Res"].cpu().numpy()
    assert np.all(np.abs(Res - oi["Res"]) <= 2 * np.spacing(np.abs(oi["Res"])) + 1e-300)
    W = mats["W"].cpu().numpy()
    g_min = oi["plan"]["g"]
    assert np.sqrt(np.sum((W - oi["W"]) ** 2)) <= delta * g_min * 1e-3
    E = mats["E"].cpu().numpy()
    assert np.sqrt(np.sum((E - oi["E"]) ** 2)) <= delta * 1e-3 + 4 * U * np.sqrt(np.sum(oi["E"] ** 2))
    Xg = Xt.cpu().numpy()
    assert np.max(np.abs(Xg - Xn)) <= 4 * U * np.max(np.abs(Xn))
    return info, oi


def test_refine_step_parity_workload0(api):
    A, X0, D0 = synth.workload0()
    _step_compare(api, A, X0, D0, 1e-14, orf.Options(), api.Options())
    _step_compare(api, A, X0, D0, 1e-14, orf.Options(slices_A=8), api.Options(slices_A=8))


@pytest.mark.parametrize("n,cond,variant", [(300, 1e4, "spd"), (257, 1e6, "indefinite")])
def test_refine_step_parity_several_tiles(api, n, cond, variant):
    A, X0, D0, lam = synth.refine_workload(n, cond, variant, case=n)
    _step_compare(api, A, X0, D0, 1e-12, orf.Options(), api.Options())


@pytest.mark.parametrize("n", [300, 1100])
def test_refine_step_parity_repeated_estimates(api, n):
    # the smallest gap of the starting estimates (Sec. 4.1, in beta) taken over an order of D
    # with exactly repeated values: the device ranks the estimates with many blocks and places
    # them by rank, ties broken by index, and the plan must match the oracle's sorted gaps
    A, X0, D0, lam = synth.refine_workload(n, 1e4, "indefinite", case=n + 7)
    D0 = D0.copy()
    D0[5::11] = D0[4::11][: len(D0[5::11])]            # exact duplicates next to each other
    D0[n // 2] = D0[3]                                  # and one far from its twin
    assert len(np.unique(D0)) < n
    _step_compare(api, A, X0, D0, 1e-12, orf.Options(), api.Options())


@pytest.mark.parametrize("xp", [3, 7])
def test_refine_step_parity_previous_study_form(api, xp):
    # X kept at xp digit planes (no truncation rule): beta = 54 - 8 xp, below 3 for xp = 7
    A, X0, D0, lam = synth.refine_workload(257, 1e6, "spd", case=257)
    _step_compare(api, A, X0, D0, 1e-12, orf.Options(x_planes=xp), api.Options(x_planes=xp))


def test_refine_step_parity_sparse_rule(api):
    # Sec. 4's sparse-matrix beta rule; k (max nonzeros in a row of A) is counted on the device
    A, X0, D0, lam = synth.banded_workload(300, 2, 12)
    info, oi = _step_compare(api, A, X0, D0, 1e-12, orf.Options(sparse_rule=True), api.Options(sparse_rule=True))
    assert info["alpha"] == oi["alpha"]


def test_refine_converges_like_the_oracle(api):
    g = G()
    A, X0, D0 = synth.workload0()
    Xh, Xl, _, _ = tr.eigvecs_dd(A, X0)
    At, Xt, Dt = g.to_dev(A), g.to_dev(X0), g.to_dev(D0)
    api.profile_read(reset=True)
    info = api.refine(At, Xt, Dt, 1e-14)
    prof = api.profile_read(reset=True)
    # every slice product of the refinement ran on the tensor cores
    assert prof["gemm_launches"] > 0 and prof["simt_launches"] == 0
    Xo, lo, oi = orf.refine(A, X0, D0, 1e-14, orf.Options())
    assert info["status"] == 0 and info["iters"] == oi["iters"]
    assert info["products"] == oi["products"]
    fe = tr.forward_error(Xh, Xl, Xt.cpu().numpy())
    assert fe <= 1e-14
    assert np.max(np.abs(Xt.cpu().numpy() - Xo)) <= 4 * U


def test_refine_fixed_slices_stagnates(api):
    g = G()
    A, X0, D0 = synth.workload0()
    At, Xt, Dt = g.to_dev(A), g.to_dev(X0), g.to_dev(D0)
    # 7 planes of A (56 bits) cannot resolve the gaps to 1e-14
    info = api.refine(At, Xt, Dt, 1e-14, api.Options(slices_A=7, max_iter=3))
    assert info["status"] in (1, 2)


def test_refine_clustered_auto(api):
    g = G()
    n = 32
    A, Q, lam = synth.symmetric_matrix(n, 1e2, 5, "clustered", cluster_pairs=2, cluster_gap=1e-10)
    X0, D0 = synth.initial_guess(Q, lam, 5, 1e-8)
    Xh, Xl, _, _ = tr.eigvecs_dd(A, X0)
    At, Xt, Dt = g.to_dev(A), g.to_dev(X0), g.to_dev(D0)
    info = api.refine(At, Xt, Dt, 1e-12, api.Options(cluster_omega=-1.0))
    assert info["status"] == 0
    X = Xt.cpu().numpy()
    ci = np.nonzero(np.diff(np.sort(lam)) < 1e-9)[0]
    for i in ci:
        assert tr.subspace_error(Xh, Xl, X, [i, i + 1]) <= 1e-12


def test_refine_rejects_bad_input(api):
    g = G()
    A, X0, D0 = synth.workload0()
    At, Xt, Dt = g.to_dev(A), g.to_dev(X0), g.to_dev(D0)
    with pytest.raises(api.FrxError) as ex:
        api.refine(At, Xt, Dt, U)
    assert ex.value.status == -3
    A2 = A.copy()
    A2[3, 5] = np.inf
    with pytest.raises(api.FrxError) as ex:
        api.refine(g.to_dev(A2), Xt, Dt, 1e-12)
    assert ex.value.status == -2
    work = api.workspace(1024)
    with pytest.raises(api.FrxError) as ex:
        api.refine(At, Xt, Dt, 1e-12, work=work)
    assert ex.value.status == -5


def test_fp64_comparator_reaches_delta():
    from paper_2602_19090_gb300 import fp64_refine
    g = G()
    A, X0, D0 = synth.workload0()
    Xh, Xl, _, _ = tr.eigvecs_dd(A, X0)
    X, lam, info = fp64_refine.refine(g.to_dev(A), g.to_dev(X0), g.to_dev(D0), 1e-14)
    assert info["status"] == "converged"
    assert tr.forward_error(Xh, Xl, X.cpu().numpy()) <= 1e-14


def test_refine_batched_matches_single(api):
    # the graph-captured batch runs the same kernels and device plans as frx_refine
    g = G()
    probs = [synth.refine_workload(nn, c, v, case=nn) for nn, c, v in
             ((40, 1e3, "spd"), (64, 1e6, "spd"), (130, 1e4, "indefinite"), (257, 1e2, "spd"), (65, 1e8, "spd"))]
    As = [g.to_dev(p[0]) for p in probs]
    Xb = [g.to_dev(p[1]) for p in probs]
    Db = [g.to_dev(p[2]) for p in probs]
    infos = api.refine_batched(As, Xb, Db, 1e-13)
    for p, A, Xg, Dg, info in zip(probs, As, Xb, Db, infos):
        Xs, Ds = g.to_dev(p[1]), g.to_dev(p[2])
        ref = api.refine(A, Xs, Ds, 1e-13)
        assert info["iters"] == ref["iters"] and info["status"] == ref["status"]
        assert info["products"] == ref["products"]
        assert np.array_equal(Xg.cpu().numpy(), Xs.cpu().numpy())
        assert np.array_equal(Dg.cpu().numpy(), Ds.cpu().numpy())


@pytest.mark.parametrize("xi,factor", [(0.0, 2.0), (1.0, 1.0)])
def test_refine_batched_forward_error(api, xi, factor):
    # Sec. 4.1 (xi = n) aims at an error of about delta (O(delta), the paper's figures);
    # the eq. proposed_beta form with xi = 1 keeps it below delta
    g = G()
    probs = [synth.refine_workload(nn, 1e3, "spd", case=7 + nn) for nn in (33, 96, 200)]
    Xs = [g.to_dev(p[1]) for p in probs]
    infos = api.refine_batched([g.to_dev(p[0]) for p in probs], Xs, [g.to_dev(p[2]) for p in probs], 1e-13,
                               api.Options(xi=xi))
    for p, X, info in zip(probs, Xs, infos):
        Xh, Xl, _, _ = tr.eigvecs_dd(p[0], p[1])
        assert info["status"] == 0
        assert tr.forward_error(Xh, Xl, X.cpu().numpy()) <= factor * 1e-13


def test_ozaki_gemm_more_than_65535_columns(api):
    # column counts beyond the 65535 limit of a grid's y dimension (slicing and recombination
    # put columns on x); small m and k keep the oracle quick
    g = G()
    m, K, n, k = 8, 40, 70000, 5
    A = synth.gemm_operand(m, K, 1.0, 320)
    B = synth.gemm_operand(K, n, 1.0, 321)
    Ch, Cl = api.ozaki_gemm(g.to_dev(A), g.to_dev(B), k, "triangular", return_lo=True)
    C_ref, o = oz.ozaki_gemm(A, B, k, "triangular")
    Ch, Cl = Ch.cpu().numpy(), Cl.cpu().numpy()
    mag = np.abs(A) @ np.abs(B)
    assert np.all(np.abs((Ch - o["hi"]) + (Cl - o["lo"])) <= mag * 2.0 ** -100)
    assert np.all(np.abs(Ch - C_ref) <= np.spacing(np.abs(C_ref)))


def test_refine_batched_more_problems_than_one_grouped_launch(api):
    # 2100 small problems: more than one chunk of grouped launches (2048); a sample of them
    # must equal single-matrix calls bit for bit
    g = G()
    rng = synth.rng(synth.seed_for(3, 77))
    sizes = rng.integers(8, 17, size=2100)
    probs = []
    for b, nn in enumerate(sizes):
        A, Q, lam = synth.symmetric_matrix(int(nn), 1e3, synth.seed_for(3, 5000 + b))
        X0, D0 = synth.initial_guess(Q, lam, synth.seed_for(3, 5000 + b))
        probs.append((A, X0, D0))
    As = [g.to_dev(p[0]) for p in probs]
    Xb = [g.to_dev(p[1]) for p in probs]
    Db = [g.to_dev(p[2]) for p in probs]
    infos = api.refine_batched(As, Xb, Db, 1e-12)
    assert all(i["status"] >= 0 for i in infos)
    for b in (0, 1, 2047, 2048, 2099):
        Xs, Ds = g.to_dev(probs[b][1]), g.to_dev(probs[b][2])
        ref = api.refine(As[b], Xs, Ds, 1e-12)
        assert infos[b]["iters"] == ref["iters"] and infos[b]["products"] == ref["products"]
        assert np.array_equal(Xb[b].cpu().numpy(), Xs.cpu().numpy())


@pytest.mark.parametrize("kind", ["banded", "random"])
def test_sparse_v_product_matches_the_dense_one(api, kind):
    # under the sparse rule, V = A X^(1) over A's nonzeros (forced: FRX_SPARSE_V=1) gives the
    # tensor-core product's exact sums bit for bit: the whole refinement returns identical X, D
    # and report
    import os
    g = G()
    if kind == "banded":
        A, X0, D0, lam = synth.banded_workload(1024, 3, 21)
    else:
        A, X0, D0, lam = synth.random_sparse_workload(768, 12, 22)
    assert int(np.max(np.count_nonzero(A, axis=1))) <= 64      # fits the ELL layout
    res = {}
    old = os.environ.get("FRX_SPARSE_V")
    try:
        for flag in ("1", "0"):
            os.environ["FRX_SPARSE_V"] = flag
            X, D = g.to_dev(X0), g.to_dev(D0)
            info = api.refine(g.to_dev(A), X, D, 1e-12, api.Options(sparse_rule=True))
            res[flag] = (X.cpu().numpy(), D.cpu().numpy(), info)
    finally:
        if old is None:
            os.environ.pop("FRX_SPARSE_V", None)
        else:
            os.environ["FRX_SPARSE_V"] = old
    assert res["1"][2]["status"] == 0
    assert np.array_equal(res["1"][0], res["0"][0]) and np.array_equal(res["1"][1], res["0"][1])
    for key in ("iters", "products", "err_est", "step", "beta", "k_V"):
        assert res["1"][2][key] == res["0"][2][key]


@pytest.mark.parametrize("kind", ["banded", "random"])
def test_sparse_v_step_matches_the_oracle(api, kind, monkeypatch):
    monkeypatch.setenv("FRX_SPARSE_V", "1")
    if kind == "banded":
        A, X0, D0, lam = synth.banded_workload(300, 2, 24)
    else:
        A, X0, D0, lam = synth.random_sparse_workload(400, 10, 23)
    _step_compare(api, A, X0, D0, 1e-12, orf.Options(sparse_rule=True), api.Options(sparse_rule=True))
