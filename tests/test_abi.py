"""The C-ABI library loads and exports every symbol include/frx.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_19090_gb300 import _lib, build_lib
    if not os.path.exists(_lib.LIB_PATH):
        build_lib.build()
    return _lib.load()


def declared():
    src = open(os.path.join(ROOT, "include", "frx.h")).read()
    return sorted(set(re.findall(r"FRX_API\s+[\w\s\*]*?\b(frx_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for required in ("frx_refine", "frx_ozaki_gemm", "frx_refine_workspace_bytes",
                     "frx_status_string", "frx_refine_step"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2602_19090_gb300 import _lib
    for name in declared():
        assert hasattr(lib, name), name
    assert sorted(declared()) == _lib.exported_names()


def test_host_only_calls(lib):
    from paper_2602_19090_gb300 import _lib
    assert lib.frx_status_string(-3) == b"delta must exceed 2^-53"
    o = _lib.Opts()
    lib.frx_default_opts(ctypes.byref(o))
    assert (o.slices_A, o.k_cap, o.max_iter, o.beta_override, o.x_planes, o.sparse_rule) == (0, 16, 10, -1, 0, 0)
    assert lib.frx_refine_workspace_bytes(0, None) == 0
    assert lib.frx_refine_workspace_bytes(64, None) > 64 * 64 * 8 * 3
    assert lib.frx_refine_workspace_bytes(12289, None) == 0
    assert lib.frx_ozaki_gemm_workspace_bytes(10, 10, 10, 17) == 0
    assert lib.frx_ozaki_gemm_workspace_bytes(10, 10, 10, 16) > 0


def test_wait_self_test_checks_its_scratch_first(lib):
    assert lib.frx_check_wait_timeout(None, 256, None) == -5
    assert lib.frx_check_wait_timeout(ctypes.c_void_p(256), 128, None) == -5


def test_tile_policy_is_host_only(lib):
    # the autotuner's switch and counters touch no device
    assert lib.frx_set_tile(3) == -1 and lib.frx_set_tile(-1) == -1
    assert lib.frx_set_tile(1) == 0
    assert lib.frx_set_tile(2) == 1
    assert lib.frx_set_tile(0) == 2
    m, d, h = ctypes.c_longlong(-1), ctypes.c_longlong(-1), ctypes.c_longlong(-1)
    assert lib.frx_tune_stats(ctypes.byref(m), ctypes.byref(d), ctypes.byref(h), 1) == 0
    assert lib.frx_tune_stats(ctypes.byref(m), ctypes.byref(d), ctypes.byref(h), 0) == 0
    assert (m.value, d.value, h.value) == (0, 0, 0)
    assert lib.frx_last_tile() == 0


def test_argument_errors_before_any_device_work(lib):
    from paper_2602_19090_gb300 import _lib
    info = _lib.Info()
    p = ctypes.c_void_p(256)   # never dereferenced: validation fails first
    st = lib.frx_refine(p, 4, p, 4, p, 4, 2.0 ** -53, None, p, 1 << 20, ctypes.byref(info), None)
    assert st == -3 and info.status == -3
    st = lib.frx_refine(None, 4, p, 4, p, 4, 1e-10, None, p, 1 << 20, None, None)
    assert st == -1
    st = lib.frx_refine(p, 3, p, 4, p, 4, 1e-10, None, p, 1 << 20, None, None)
    assert st == -1
    st = lib.frx_refine(p, 4, p, 4, p, 4, 1e-10, None, None, 0, None, None)
    assert st == -5
    o = _lib.Opts()
    lib.frx_default_opts(ctypes.byref(o))
    o.x_planes = 8                  # more planes than FP64 width needs (7 x 8 bits)
    st = lib.frx_refine(p, 4, p, 4, p, 4, 1e-10, ctypes.byref(o), p, 1 << 20, None, None)
    assert st == -1
    lib.frx_default_opts(ctypes.byref(o))
    o.sparse_rule = 2
    st = lib.frx_refine(p, 4, p, 4, p, 4, 1e-10, ctypes.byref(o), p, 1 << 20, None, None)
    assert st == -1
    st = lib.frx_ozaki_gemm(p, 4, p, 4, p, 4, None, 4, 4, 4, 0, 0, p, 1 << 20, None)
    assert st == -1


def test_empty_sizes_are_refused_before_any_device_work(lib):
    # n = 0 (or m, n, k = 0 for a product) is an argument error, with no device work and no
    # scratch requirement
    p = ctypes.c_void_p(256)
    assert lib.frx_refine(p, 4, p, 4, p, 0, 1e-10, None, p, 1 << 20, None, None) == -1
    assert lib.frx_refine(p, 4, p, 4, p, -1, 1e-10, None, p, 1 << 20, None, None) == -1
    N = None
    assert lib.frx_refine_step(p, 4, p, 4, p, 0, 1e-10, None, 0.0, p, 1 << 20, None,
                               N, N, N, N, N, N, N, None) == -1
    for m, n, k in ((0, 8, 8), (8, 0, 8), (8, 8, 0)):
        assert lib.frx_ozaki_gemm(p, 8, p, 8, p, 8, None, m, n, k, 4, 0, p, 1 << 30, None) == -1
    assert lib.frx_refine_workspace_bytes(0, None) == 0
    assert lib.frx_ozaki_gemm_workspace_bytes(0, 8, 8, 4) == 0


def test_group_size_keeps_sums_exact(lib):
    # groups of gs anti-diagonals: max|S_t| * 2^(8 (gs - 1)) * 256/255 < 2^62, where
    # max|S_t| = pairs * K * 128^2 (8-bit digits)
    for kL, kR, T, K in ((8, 6, 9, 64), (16, 8, 17, 12288), (16, 16, 32, 65536), (3, 3, 4, 5)):
        gs = lib.frx_group_size(kL, kR, T, K)
        pmax = max(sum(1 for r in range(1, kL + 1) if 1 <= t - r <= kR and t <= T)
                   for t in range(2, min(T, kL + kR) + 1))
        smax = pmax * K * 16384
        assert smax * 2 ** (8 * (gs - 1)) * 256 / 255 < 2 ** 62
        assert smax * 2 ** (8 * gs) * 256 / 255 >= 2 ** 61    # not needlessly small


def test_batched_argument_errors_before_any_device_work(lib):
    import ctypes as C
    p = C.c_void_p(256)
    P1 = C.c_void_p * 1
    I1 = C.c_int64 * 1
    A, ld, n = P1(256), I1(4), I1(4)
    work, big = p, 1 << 20

    def call(A=A, lda=ld, X=A, ldx=ld, D=A, n=n, count=1, delta=1e-10, work=work, wb=big):
        return lib.frx_refine_batched(A, lda, X, ldx, D, n, count, delta, None, work, wb, None, None)

    assert call(count=0) == -1 and call(count=-1) == -1
    assert call(A=None) == -1 and call(n=None) == -1
    assert call(A=P1(None)) == -1
    assert call(lda=I1(3)) == -1 and call(n=I1(0)) == -1
    assert call(delta=2.0 ** -53) == -3
    assert call(n=I1(12289), lda=I1(12289), ldx=I1(12289)) == -7
    # scratch: NULL, misaligned, one byte short of the documented size
    need = lib.frx_refine_batched_workspace_bytes(n, 1, None)
    assert need > 0 and lib.frx_refine_batched_workspace_bytes(n, 0, None) == 0
    assert call(work=None, wb=0) == -5
    assert call(work=C.c_void_p(256 + 8)) == -5
    assert call(wb=need - 1) == -5


def test_ozaki_gemm_limits_before_any_device_work(lib):
    import ctypes as C
    p = C.c_void_p(256)
    # the allocation-free form: m, n, k <= 512 and slices <= 8
    assert lib.frx_ozaki_gemm_static(p, 513, p, 513, p, 513, None, 513, 4, 4, 4, 0, None) == -7
    assert lib.frx_ozaki_gemm_static(p, 8, p, 8, p, 8, None, 8, 8, 8, 9, 0, None) == -7
    assert lib.frx_ozaki_gemm_static(p, 8, p, 8, p, 8, None, 0, 8, 8, 4, 0, None) == -1
    # the general form: slices 1..16, a known mode, k <= 65536, enough scratch
    assert lib.frx_ozaki_gemm(p, 8, p, 8, p, 8, None, 8, 8, 8, 17, 0, p, 1 << 30, None) == -1
    assert lib.frx_ozaki_gemm(p, 8, p, 8, p, 8, None, 8, 8, 8, 4, 2, p, 1 << 30, None) == -1
    assert lib.frx_ozaki_gemm(p, 8, p, 65537, p, 8, None, 8, 8, 65537, 4, 0, p, 1 << 30, None) == -7
    need = lib.frx_ozaki_gemm_workspace_bytes(8, 8, 8, 4)
    assert lib.frx_ozaki_gemm(p, 8, p, 8, p, 8, None, 8, 8, 8, 4, 0, p, need - 1, None) == -5


def test_bit_level_calls_check_their_arguments(lib):
    import ctypes as C
    p, e = C.c_void_p(256), C.c_void_p(512)
    assert lib.frx_exponents(p, 4, 4, 4, 2, e, p, 1 << 20, None) == -1      # axis 0 or 1
    assert lib.frx_exponents(p, 3, 4, 4, 0, e, p, 1 << 20, None) == -1      # ld < rows
    assert lib.frx_slice_planes(p, 4, 4, 4, 0, e, 17, p, 1 << 10, 8, None) == -1   # k <= 16
    assert lib.frx_slice_planes(p, 4, 4, 4, 0, e, 4, p, 1 << 10, 7, None) == -1    # pitch % 8
    assert lib.frx_plane_products(p, 1024, p, 1024, 8, 4, 4, 4, 0, 4, 5, p, None) == -1  # kL >= 1


def test_binding_empty_batch_is_a_no_op(lib):
    from paper_2602_19090_gb300 import api
    assert api.refine_batched([], [], [], 1e-12) == []
    with pytest.raises(ValueError):
        api.refine_batched([], [None], [], 1e-12)


def test_workspace_sizes_grow_with_the_problem(lib):
    import ctypes as C
    from paper_2602_19090_gb300 import _lib
    o = _lib.Opts()
    lib.frx_default_opts(C.byref(o))
    sizes = [lib.frx_refine_workspace_bytes(n, C.byref(o)) for n in (1, 2, 63, 64, 65, 1000, 4096, 12288)]
    assert all(b > 0 for b in sizes)
    assert sizes == sorted(sizes) and len(set(sizes[3:])) == len(sizes[3:])
    o.k_cap = 8                       # fewer planes of A: less scratch
    assert lib.frx_refine_workspace_bytes(4096, C.byref(o)) < sizes[6]
    g = [lib.frx_ozaki_gemm_workspace_bytes(300, 200, 500, k) for k in range(1, 17)]
    assert all(b > 0 for b in g) and g == sorted(g)
    I = C.c_int64 * 3
    one = lib.frx_refine_batched_workspace_bytes(I(100, 0, 0), 1, None)
    three = lib.frx_refine_batched_workspace_bytes(I(100, 200, 50), 3, None)
    assert 0 < one < three
    assert lib.frx_refine_batched_workspace_bytes(I(100, 12289, 50), 3, None) == 0


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    # no CPU fallback: without the CUDA library every entry point of the binding raises
    from paper_2602_19090_gb300 import _lib, api
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libfrx.so"))
    with pytest.raises(RuntimeError, match="library missing"):
        _lib.load()
    with pytest.raises(RuntimeError, match="library missing"):
        api.refine_batched([], [], [], 1e-12)
    with pytest.raises(RuntimeError, match="library missing"):
        api.last_tile()
