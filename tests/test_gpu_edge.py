"""Edge cases of the CUDA path: the smallest problems, degenerate matrices, the largest
sizes the library accepts, and the int64-group form of the slice products."""
import numpy as np
import pytest

from oracle import ozaki as oz
from oracle import refine as orf
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


@pytest.mark.parametrize("n", [1, 2, 3])
def test_refine_smallest_problems_match_the_oracle(api, n):
    g = G()
    A, Q, lam = synth.symmetric_matrix(n, 1e2, 40 + n)
    X0, D0 = synth.initial_guess(Q, lam, 40 + n)
    Xo, lo, oi = orf.refine(A, X0, D0, 1e-13, orf.Options())
    Xt, Dt = g.to_dev(X0), g.to_dev(D0)
    info = api.refine(g.to_dev(A), Xt, Dt, 1e-13)
    assert info["status"] == 0 and oi["status"] == "converged"
    assert info["iters"] == oi["iters"]
    assert np.max(np.abs(Xt.cpu().numpy() - Xo)) <= 4 * U * np.max(np.abs(Xo))


def test_diagonal_matrix_identity_start_is_a_fixed_point(api):
    # A = diag(d) with distinct d: X = I, lambda = d are exact; one step must return them
    g = G()
    n = 70
    d = np.arange(1, n + 1, dtype=np.float64)[::-1] * 0.75
    A = np.diag(d)
    info, mats = api.refine_step(g.to_dev(A), g.to_dev(np.eye(n)), g.to_dev(d.copy()), 1e-13)
    assert np.array_equal(mats["X1"].cpu().numpy(), np.eye(n))
    Xt = g.to_dev(np.eye(n))
    Dt = g.to_dev(d.copy())
    info = api.refine(g.to_dev(A), Xt, Dt, 1e-13)
    assert info["status"] == 0
    assert np.array_equal(Xt.cpu().numpy(), np.eye(n))
    assert np.array_equal(Dt.cpu().numpy(), d)


def test_zero_matrix_is_handled(api):
    # all eigenvalues equal (zero): every pair is a cluster pair (up to 64 per column are kept
    # on the device), no gap exists, so no estimate can certify convergence: the iteration runs
    # to its limit and leaves the exact eigenvectors unchanged
    g = G()
    n = 16
    Xt = g.to_dev(np.eye(n))
    Dt = g.to_dev(np.zeros(n))
    info = api.refine(g.to_dev(np.zeros((n, n))), Xt, Dt, 1e-12, api.Options(max_iter=3))
    assert info["status"] == 1
    assert np.array_equal(Xt.cpu().numpy(), np.eye(n))


def test_largest_accepted_size(api):
    # n = 12288 (the library's limit): diagonal A with distinct entries and a perturbed
    # identity start converge to the identity (the exact eigenvectors)
    import torch
    g = G()
    n = 12288
    d = np.linspace(1.0, 2.0, n)
    dev = g.dev()
    A = torch.diag(torch.from_numpy(d)).to(dev)
    rng = synth.rng(synth.seed_for(2, 12288))
    X = torch.eye(n, dtype=torch.float64, device=dev) + torch.from_numpy(
        rng.standard_normal((n, n)) * (1e-9 / np.sqrt(n))).to(dev)
    D = torch.from_numpy(d * (1.0 + 1e-9 * rng.standard_normal(n))).to(dev)
    info = api.refine(A, X, D, 1e-12)
    assert info["status"] == 0
    err = (X.abs() - torch.eye(n, dtype=torch.float64, device=dev)).abs().max().item()
    assert err <= 1e-12
    dd = torch.from_numpy(d).to(dev)
    assert ((D - dd).abs() <= 2 * U * dd.abs()).all()


def test_ozaki_gemm_longest_inner_dimension_int64_groups(api):
    # k = 65536 (the limit) with 8 planes, all pairs: up to 8 pairs per anti-diagonal make
    # 8 * 65536 * 2^14 = 2^33, beyond int32, so the int64 Horner groups are used
    g = G()
    m, K, n, k = 136, 65536, 130, 8
    A = synth.gemm_operand(m, K, 1.0, 330)
    B = synth.gemm_operand(K, n, 1.0, 331)
    Ch, Cl = api.ozaki_gemm(g.to_dev(A), g.to_dev(B), k, "full", return_lo=True)
    C_ref, o = oz.ozaki_gemm(A, B, k, "full")
    Ch, Cl = Ch.cpu().numpy(), Cl.cpu().numpy()
    mag = np.abs(A) @ np.abs(B)
    assert np.all(np.abs((Ch - o["hi"]) + (Cl - o["lo"])) <= mag * 2.0 ** -100)
    assert np.all(np.abs(Ch - C_ref) <= np.spacing(np.abs(C_ref)))


def test_bounded_wait_reports_timeout_and_the_context_survives(api):
    # a device wait on an mbarrier that nothing completes gives up after its limit (2 s),
    # the call reports FRX_E_TIMEOUT, and the next call on the same context works
    import ctypes
    import time

    import torch
    from paper_2602_19090_gb300 import _lib
    g = G()
    lib = _lib.load()
    work = api.workspace(256, g.dev())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    t0 = time.perf_counter()
    st = lib.frx_check_wait_timeout(ctypes.c_void_p(work.data_ptr()), 256, stream)
    elapsed = time.perf_counter() - t0
    assert st == -6
    assert 1.5 < elapsed < 60
    A = synth.gemm_operand(70, 90, 1.0, 340)
    B = synth.gemm_operand(90, 50, 1.0, 341)
    C = api.ozaki_gemm(g.to_dev(A), g.to_dev(B), 8, "full").cpu().numpy()
    C_ref, _ = oz.ozaki_gemm(A, B, 8, "full")
    assert np.all(np.abs(C - C_ref) <= np.spacing(np.abs(C_ref)))


def test_batched_calls_from_two_threads(api):
    # two host threads run batched refinements on the same device at once (each with its
    # own problems and scratch): the calls are serialised inside the library and each
    # result equals the same call made alone
    import threading

    g = G()
    sets = []
    for base in (0, 100):
        probs = [synth.refine_workload(nn, 1e3, "spd", case=base + nn) for nn in (40, 75, 130)]
        sets.append(probs)
    alone = []
    for probs in sets:
        Xs = [g.to_dev(p[1]) for p in probs]
        api.refine_batched([g.to_dev(p[0]) for p in probs], Xs, [g.to_dev(p[2]) for p in probs], 1e-12)
        alone.append([x.cpu().numpy() for x in Xs])
    outs = [None, None]
    errs = []

    def run(k):
        try:
            import torch
            torch.cuda.set_device(0)
            probs = sets[k]
            Xs = [g.to_dev(p[1]) for p in probs]
            api.refine_batched([g.to_dev(p[0]) for p in probs], Xs, [g.to_dev(p[2]) for p in probs], 1e-12)
            torch.cuda.synchronize()
            outs[k] = [x.cpu().numpy() for x in Xs]
        except Exception as e:   # reported below
            errs.append(e)

    th = [threading.Thread(target=run, args=(k,)) for k in (0, 1)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    for k in (0, 1):
        for a, b in zip(outs[k], alone[k]):
            assert np.array_equal(a, b)


def test_batched_plan_reuse_sees_new_data_and_a_clobbered_scratch(api):
    # a repeated batched call with the same pointers, sizes and options reuses its launch plan
    # (recorded stages, argument tables, iteration graph): with the scratch overwritten in
    # between it must give the same bits, and with new data in the same buffers the result of
    # the new data (equal to single-matrix calls on it)
    import torch
    g = G()
    probs = [synth.refine_workload(nn, 1e3, "spd", case=600 + nn) for nn in (50, 90, 140)]
    As = [g.to_dev(p[0]) for p in probs]
    Xs = [api.colmajor(g.to_dev(p[1]))[0] for p in probs]   # passed without copies: same pointers
    Ds = [g.to_dev(p[2]) for p in probs]
    X0s = [x.clone() for x in Xs]
    D0s = [d.clone() for d in Ds]
    import ctypes as C
    o = api.Options().to_c()
    nn = (C.c_int64 * 3)(*[p[0].shape[0] for p in probs])
    work = api.workspace(api._lib.load().frx_refine_batched_workspace_bytes(nn, 3, C.byref(o)), g.dev())
    api.refine_batched(As, Xs, Ds, 1e-12, work=work)
    first = [x.cpu().numpy() for x in Xs]
    work.fill_(255)
    for x, x0, d, d0 in zip(Xs, X0s, Ds, D0s):
        x.copy_(x0)
        d.copy_(d0)
    api.refine_batched(As, Xs, Ds, 1e-12, work=work)
    for a, b in zip(first, Xs):
        assert np.array_equal(a, b.cpu().numpy())
    # new starting eigenpairs in the same buffers
    for k, (x, d) in enumerate(zip(Xs, Ds)):
        A, Q, lam = synth.symmetric_matrix(probs[k][0].shape[0], 1e3, synth.seed_for(2, 600 + probs[k][0].shape[0]))
        X1, D1 = synth.initial_guess(Q, lam, 77 + k, rel=1e-7)
        x.copy_(torch.from_numpy(X1))
        d.copy_(torch.from_numpy(D1))
    starts = [(x.clone(), d.clone()) for x, d in zip(Xs, Ds)]
    api.refine_batched(As, Xs, Ds, 1e-12, work=work)
    for A, (x0, d0), x in zip(As, starts, Xs):
        xs, ds = x0.clone(), d0.clone()
        api.refine(A, xs, ds, 1e-12)
        assert np.array_equal(xs.cpu().numpy(), x.cpu().numpy())
