"""The tcgen05 slice-product kernel against the CUDA-core kernel, bit for bit (GB300)."""
import os

import numpy as np
import pytest

from paper_2602_19090_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_19090_gb300 import api as a
    return a


def _both(api, Lp, Rp, K, kL, kR, T):
    import torch
    old = os.environ.get("FRX_GEMM")
    try:
        # the profile counts each product that ran on the CUDA cores
        api.profile_read(reset=True)
        os.environ["FRX_GEMM"] = "simt"
        ref, gs = api.plane_products(Lp, Rp, K, kL, kR, T)
        assert api.profile_read(reset=True)["simt_launches"] == 1
        os.environ["FRX_GEMM"] = "tc"
        got, gs2 = api.plane_products(Lp, Rp, K, kL, kR, T)
        torch.cuda.synchronize()
        assert api.profile_read(reset=True)["simt_launches"] == 0
    finally:
        if old is None:
            os.environ.pop("FRX_GEMM", None)
        else:
            os.environ["FRX_GEMM"] = old
    assert gs == gs2
    return ref.cpu().numpy(), got.cpu().numpy()


@pytest.mark.parametrize("m,n,K,kL,kR,T", [
    (128, 128, 64, 1, 1, 2),          # one tile, one k-block, one product
    (128, 128, 128, 2, 2, 4),
    (200, 150, 300, 4, 3, 5),         # ragged tiles and K
    (256, 384, 2048, 3, 3, 4),        # exactly one chunk per pair
    (130, 260, 5000, 5, 4, 6),        # chunks split inside pairs, several groups
    (1, 1, 1, 2, 2, 4),
])
def test_tc_matches_simt(api, m, n, K, kL, kR, T):
    from tests import gpu_util as g
    L = synth.gemm_operand(m, K, 2.0, 500 + m)
    R = synth.gemm_operand(K, n, 2.0, 600 + n)
    Lt, Rt = g.to_dev(L), g.to_dev(R)
    Lp = api.slice_planes(Lt, 0, api.exponents(Lt, 0), kL)
    Rp = api.slice_planes(Rt, 1, api.exponents(Rt, 1), kR)
    ref, got = _both(api, Lp, Rp, K, kL, kR, T)
    assert np.array_equal(ref, got)


def test_tc_worst_case_digits(api):
    # every digit +128 (all-ones matrix): FP32 chunk sums reach 1024 * 2^14 = 2^24 exactly
    from tests import gpu_util as g
    K = 4096 + 64
    Lt = g.to_dev(np.ones((256, K)))
    Lp = api.slice_planes(Lt, 0, api.exponents(Lt, 0), 3)
    ref, got = _both(api, Lp, Lp.clone(), K, 3, 3, 6)
    assert np.array_equal(ref, got)
    # only plane 1 is nonzero (digit 128), so group 0 holds S_2 shifted to its last t
    gs = api.group_size(3, 3, 6, K)
    t_last = min(2 + gs - 1, 6)
    assert ref[0, 0, 0] == 128 * 128 * K * 2 ** (8 * (t_last - 2))


@pytest.mark.parametrize("m,k,n,slices,mode", [(300, 513, 260, 6, "full"), (1024, 2048, 512, 8, "triangular"),
                                               (129, 4100, 257, 5, "full")])
def test_ozaki_gemm_tensor_core_equals_cuda_core(api, m, k, n, slices, mode):
    # exercises the 128 x 256 tiles with one int32 plane per anti-diagonal
    import torch
    from tests import gpu_util as g
    A = g.to_dev(synth.gemm_operand(m, k, 2.0, 700 + m))
    B = g.to_dev(synth.gemm_operand(k, n, 2.0, 800 + n))
    old = os.environ.get("FRX_GEMM")
    try:
        os.environ["FRX_GEMM"] = "simt"
        ch0, cl0 = api.ozaki_gemm(A, B, slices, mode, return_lo=True)
        os.environ["FRX_GEMM"] = "tc"
        ch1, cl1 = api.ozaki_gemm(A, B, slices, mode, return_lo=True)
        torch.cuda.synchronize()
    finally:
        if old is None:
            os.environ.pop("FRX_GEMM", None)
        else:
            os.environ["FRX_GEMM"] = old
    assert torch.equal(ch0, ch1) and torch.equal(cl0, cl1)


@pytest.mark.parametrize("m,K,n,k,mode", [(300, 65536, 260, 8, "full"),     # 4 exact chunks of 16384
                                          (200, 30000, 130, 6, "triangular"),   # few tiles: more chunks
                                          (129, 65536, 257, 16, "full")])       # 16 planes, ragged
def test_split_k_matches_the_int64_register_kernel(api, m, K, n, k, mode):
    # long inner dimensions make the anti-diagonal sums exceed int32: split-K (int32 chunks added
    # to int64 Horner groups by atomics) and the int64-register kernel give the same bits
    import torch
    from tests import gpu_util as g
    A = g.to_dev(synth.gemm_operand(m, K, 1.0, 800 + m))
    B = g.to_dev(synth.gemm_operand(K, n, 1.0, 801 + n))
    out = {}
    old = os.environ.get("FRX_SPLITK")
    try:
        for flag in ("1", "0"):
            os.environ["FRX_SPLITK"] = flag
            Ch, Cl = api.ozaki_gemm(A, B, k, mode, return_lo=True)
            torch.cuda.synchronize()
            out[flag] = (Ch.cpu().numpy(), Cl.cpu().numpy(), api.last_tile())
    finally:
        if old is None:
            os.environ.pop("FRX_SPLITK", None)
        else:
            os.environ["FRX_SPLITK"] = old
    assert out["1"][2] == "128x256" and out["0"][2] == "128x128"
    assert np.array_equal(out["1"][0], out["0"][0]) and np.array_equal(out["1"][1], out["0"][1])
