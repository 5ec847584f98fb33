"""The scratch-free Ozaki product (frx_ozaki_gemm_static) against frx_ozaki_gemm.

frx_ozaki_gemm_static exists for callers that cannot allocate device memory, such as a
plugin inside a framework that has reserved all device memory for its own allocator.
Its scratch is a fixed array inside the library, shared by every call.  These tests
call both entry points through the C ABI on the same inputs and require the same
product, bit for bit (both run the same deterministic path), on calls in a row with
different shapes (each later call runs on the scratch the one before left behind),
up to the largest accepted shape.  Free device memory is unchanged across a call once
the array is in place: the entry point allocates nothing.
"""
import ctypes

import numpy as np
import pytest

from paper_2602_19090_gb300 import synth

pytestmark = pytest.mark.gpu

STATIC_BYTES = 24 * 1024 * 1024 + 64 * 1024   # the library's fixed scratch array


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_19090_gb300 import _lib, api
    return torch, _lib.load(), api


def _operands(torch, api, m, k, n, seed):
    A = synth.gemm_operand(m, k, 2.0, seed)
    B = synth.gemm_operand(k, n, 2.0, seed + 1)
    Ad, lda, _ = api.colmajor(torch.from_numpy(A).cuda())
    Bd, ldb, _ = api.colmajor(torch.from_numpy(B).cuda())
    return A, B, Ad, lda, Bd, ldb


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_static_scratch_matches_caller_scratch_in_a_row(env):
    torch, lib, api = env
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # the last case is the largest accepted shape: the one whose workspace comes closest to
    # the fixed array
    cases = ((300, 257, 190, 6, 0, 900), (512, 512, 64, 8, 1, 910), (512, 512, 512, 8, 0, 920))
    for (m, k, n, slices, mode, seed) in cases:
        need = lib.frx_ozaki_gemm_workspace_bytes(m, n, k, slices)
        assert 0 < need <= STATIC_BYTES
        _, _, Ad, lda, Bd, ldb = _operands(torch, api, m, k, n, seed)
        ref_h, ref_l = api.empty_colmajor(m, n), api.empty_colmajor(m, n)
        got_h, got_l = api.empty_colmajor(m, n), api.empty_colmajor(m, n)
        work = api.workspace(need)
        st = lib.frx_ozaki_gemm(_p(Ad), lda, _p(Bd), ldb, _p(ref_h), m, _p(ref_l), m, n, k,
                                slices, mode, _p(work), work.numel(), stream)
        assert st == 0
        st = lib.frx_ozaki_gemm_static(_p(Ad), lda, _p(Bd), ldb, _p(got_h), m, _p(got_l), m, n, k,
                                       slices, mode, stream)
        assert st == 0
        torch.cuda.synchronize()
        assert np.array_equal(got_h.cpu().numpy(), ref_h.cpu().numpy())
        assert np.array_equal(got_l.cpu().numpy(), ref_l.cpu().numpy())


def test_static_scratch_call_allocates_nothing(env):
    torch, lib, api = env
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    m = k = n = 512
    _, _, Ad, lda, Bd, ldb = _operands(torch, api, m, k, n, 930)
    C, C_lo = api.empty_colmajor(m, n), api.empty_colmajor(m, n)

    def call():
        st = lib.frx_ozaki_gemm_static(_p(Ad), lda, _p(Bd), ldb, _p(C), m, _p(C_lo), m, n, k, 8, 0, stream)
        torch.cuda.synchronize()
        assert st == 0

    call()   # loads the array (first call on this device in a fresh process)
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        call()
    free1, _ = torch.cuda.mem_get_info()
    # a device allocation of the 24 MiB workspace (or any cudaMalloc: 2 MiB pages) would show
    assert free1 == free0


def test_static_scratch_rejects_sizes_beyond_its_limit(env):
    torch, lib, api = env
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    x = api.empty_colmajor(600, 600)
    for (m, n, k, slices) in ((513, 8, 8, 2), (8, 513, 8, 2), (8, 8, 513, 2), (8, 8, 8, 9)):
        st = lib.frx_ozaki_gemm_static(_p(x), 600, _p(x), 600, _p(x), 600, None, m, n, k,
                                       slices, 0, stream)
        assert st == -7
