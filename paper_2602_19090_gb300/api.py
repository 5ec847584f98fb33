"""Thin torch binding of the frx C ABI: argument marshalling only.

Every call runs the CUDA library; tensors must be float64 CUDA tensors.  Matrices
are passed column-major: a tensor whose storage is column-major (stride (1, ld))
is passed as-is, any other layout is copied into a column-major buffer (and
copied back for in/out arguments).
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import torch

from . import _lib

STATUS = {0: "converged", 1: "max_iter", 2: "stagnated"}
MODES = {"full": 0, "triangular": 1}


class FrxError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.load().frx_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


@dataclasses.dataclass
class Options:
    slices_A: int = 0
    xi: float = 1.0              # <= 0: xi = n (the Sec. 4.1 "n delta" form)
    beta_ceil: bool = False
    theory_alpha: bool = False
    beta_override: int = -1
    k_cap: int = 16
    max_iter: int = 10
    xi_stop: float = 0.0
    cluster_omega: float = 0.0   # < 0: automatic Ogita-Aishima threshold
    x_planes: int = 0            # > 0: X kept at x_planes digit planes (previous-study form)
    sparse_rule: bool = False    # the sparse-matrix beta rule (k = max nonzeros in a row of A)

    def to_c(self) -> _lib.Opts:
        return _lib.Opts(self.slices_A, self.xi, int(self.beta_ceil), int(self.theory_alpha),
                         self.beta_override, self.k_cap, self.max_iter, self.xi_stop,
                         self.cluster_omega, self.x_planes, int(self.sparse_rule))


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _check(st, where, soft_ok=True):
    if st < 0 or (st > 0 and not soft_ok):
        raise FrxError(st, where)
    return st


def _f64_cuda(t, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise TypeError(f"{name} must be a float64 CUDA tensor")


def colmajor(t: torch.Tensor):
    """(tensor, ld, copied): a column-major view of the matrix t."""
    if t.dim() == 2 and t.stride(0) == 1 and t.stride(1) >= max(1, t.shape[0]):
        return t, t.stride(1), False
    c = t.t().contiguous().t()
    return c, max(1, c.shape[0]), True


def symmetric_colmajor(A: torch.Tensor):
    """(tensor, ld, copied) for a symmetric matrix: a contiguous row-major square matrix is
    passed as it is, since A = A^T makes its row-major layout the column-major one."""
    if A.dim() == 2 and A.shape[0] == A.shape[1] and A.is_contiguous():
        return A, max(1, A.shape[1]), False
    return colmajor(A)


def empty_colmajor(m, n, device="cuda"):
    return torch.empty((n, m), dtype=torch.float64, device=device).t()


def workspace(nbytes: int, device="cuda") -> torch.Tensor:
    return torch.empty(int(nbytes), dtype=torch.uint8, device=device)


def refine_workspace_bytes(n: int, opts: Options | None = None) -> int:
    o = (opts or Options()).to_c()
    return _lib.load().frx_refine_workspace_bytes(n, C.byref(o))


def refine(A, X, D, delta, opts: Options | None = None, work=None, stream=None):
    """In-place refinement of (X, D); returns the frx_info report as a dict."""
    lib = _lib.load()
    for t, nm in ((A, "A"), (X, "X"), (D, "D")):
        _f64_cuda(t, nm)
    n = A.shape[0]
    o = (opts or Options()).to_c()
    Ac, lda, _ = symmetric_colmajor(A)
    Xc, ldx, xcopy = colmajor(X)
    if work is None:
        work = workspace(lib.frx_refine_workspace_bytes(n, C.byref(o)), A.device)
    info = _lib.Info()
    st = lib.frx_refine(_ptr(Ac), lda, _ptr(Xc), ldx, _ptr(D), n, float(delta), C.byref(o),
                        _ptr(work), work.numel(), C.byref(info), _stream(stream))
    _check(st, "frx_refine")
    if xcopy:
        X.copy_(Xc)
    d = info.as_dict()
    d["status_name"] = STATUS.get(st, str(st))
    return d


def refine_batched(As, Xs, Ds, delta, opts: Options | None = None, work=None, stream=None):
    """Batched in-place refinement of independent problems; returns a list of info dicts
    (an empty list for an empty batch, which the library is not called for)."""
    lib = _lib.load()
    count = len(As)
    if not (count == len(Xs) == len(Ds)):
        raise ValueError("refine_batched: As, Xs and Ds must have the same length")
    if count == 0:
        return []
    o = (opts or Options()).to_c()
    cols = [symmetric_colmajor(A) for A in As]
    xcols = [colmajor(X) for X in Xs]
    for t in list(As) + list(Xs) + list(Ds):
        _f64_cuda(t, "batched operand")
    P = C.c_void_p * count
    I64 = C.c_int64 * count
    n = I64(*[A.shape[0] for A in As])
    Ap = P(*[c[0].data_ptr() for c in cols])
    lda = I64(*[c[1] for c in cols])
    Xp = P(*[c[0].data_ptr() for c in xcols])
    ldx = I64(*[c[1] for c in xcols])
    Dp = P(*[D.data_ptr() for D in Ds])
    if work is None:
        work = workspace(lib.frx_refine_batched_workspace_bytes(n, count, C.byref(o)), As[0].device)
    infos = (_lib.Info * count)()
    st = lib.frx_refine_batched(Ap, lda, Xp, ldx, Dp, n, count, float(delta), C.byref(o), _ptr(work),
                                work.numel(), infos, _stream(stream))
    _check(st, "frx_refine_batched")
    for (Xc, _, copied), X in zip(xcols, Xs):
        if copied:
            X.copy_(Xc)
    out = []
    for i in range(count):
        d = infos[i].as_dict()
        d["status_name"] = STATUS.get(d["status"], str(d["status"]))
        out.append(d)
    return out


def refine_step(A, X, D, delta, opts: Options | None = None, omega_prev: float = 0.0,
                intermediates: bool = True, work=None, stream=None):
    """One iteration; returns (info, dict of intermediates as row-major tensors)."""
    lib = _lib.load()
    n = A.shape[0]
    o = (opts or Options()).to_c()
    Ac, lda, _ = symmetric_colmajor(A)
    Xc, ldx, xcopy = colmajor(X)
    if work is None:
        work = workspace(lib.frx_refine_workspace_bytes(n, C.byref(o)), A.device)
    names = ("X1", "Vh", "Vl", "Res", "W", "E")
    mats = {k: empty_colmajor(n, n, A.device) for k in names} if intermediates else {}
    r = torch.empty(n, dtype=torch.float64, device=A.device) if intermediates else None
    info = _lib.Info()
    st = lib.frx_refine_step(_ptr(Ac), lda, _ptr(Xc), ldx, _ptr(D), n, float(delta), C.byref(o),
                             float(omega_prev), _ptr(work), work.numel(), C.byref(info),
                             *[_ptr(mats.get(k)) for k in names], _ptr(r), _stream(stream))
    _check(st, "frx_refine_step")
    if xcopy:
        X.copy_(Xc)
    out = dict(mats)
    if r is not None:
        out["r"] = r
    return info.as_dict(), out


def ozaki_gemm_workspace_bytes(m: int, n: int, k: int, slices: int) -> int:
    return _lib.load().frx_ozaki_gemm_workspace_bytes(m, n, k, slices)


def ozaki_gemm(A, B, slices: int, mode: str = "full", return_lo: bool = False, work=None,
               stream=None):
    """C = A B by the Ozaki scheme with `slices` digit planes per operand."""
    lib = _lib.load()
    _f64_cuda(A, "A")
    _f64_cuda(B, "B")
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    Ac, lda, _ = colmajor(A)
    Bc, ldb, _ = colmajor(B)
    Cm = empty_colmajor(m, n, A.device)
    Cl = empty_colmajor(m, n, A.device) if return_lo else None
    if work is None:
        work = workspace(lib.frx_ozaki_gemm_workspace_bytes(m, n, k, slices), A.device)
    st = lib.frx_ozaki_gemm(_ptr(Ac), lda, _ptr(Bc), ldb, _ptr(Cm), m, _ptr(Cl), m, n, k,
                            int(slices), MODES[mode], _ptr(work), work.numel(), _stream(stream))
    _check(st, "frx_ozaki_gemm", soft_ok=False)
    return (Cm, Cl) if return_lo else Cm


def exponents(M, axis: int, stream=None):
    lib = _lib.load()
    Mc, ld, _ = colmajor(M)
    rows, cols = M.shape
    e = torch.empty(rows if axis == 0 else cols, dtype=torch.int32, device=M.device)
    work = workspace(lib.frx_exponents_workspace_bytes(rows), M.device)
    st = lib.frx_exponents(_ptr(Mc), ld, rows, cols, axis, _ptr(e), _ptr(work), work.numel(),
                           _stream(stream))
    _check(st, "frx_exponents", soft_ok=False)
    return e


def slice_planes(M, axis: int, e, k: int, pitch: int | None = None, stream=None):
    """bf16 digit planes as a uint16 tensor of shape (k, lines, pitch)."""
    lib = _lib.load()
    Mc, ld, _ = colmajor(M)
    rows, cols = M.shape
    lines, other = (rows, cols) if axis == 0 else (cols, rows)
    pitch = pitch or (other + 63) // 64 * 64
    planes = torch.empty((k, lines, pitch), dtype=torch.int16, device=M.device)
    st = lib.frx_slice_planes(_ptr(Mc), ld, rows, cols, axis, _ptr(e), k, _ptr(planes),
                              lines * pitch, pitch, _stream(stream))
    _check(st, "frx_slice_planes", soft_ok=False)
    return planes


def group_size(kL, kR, T, K):
    return _lib.load().frx_group_size(kL, kR, T, K)


def plane_products(Lp, Rp, K, kL, kR, T, stream=None):
    """Exact grouped slice products of plane stacks from ``slice_planes``."""
    lib = _lib.load()
    _, m, pitch = Lp.shape
    _, n, pitch2 = Rp.shape
    assert pitch == pitch2
    gs = lib.frx_group_size(kL, kR, T, K)
    if gs < 0:
        raise FrxError(gs, "frx_group_size")
    tmax = min(T, kL + kR)
    groups = (tmax - 1 + gs - 1) // gs
    out = torch.zeros((max(groups, 1), n, m), dtype=torch.int64, device=Lp.device)
    st = lib.frx_plane_products(_ptr(Lp), m * pitch, _ptr(Rp), n * pitch, pitch, m, n, K, kL, kR,
                                T, _ptr(out), _stream(stream))
    _check(st, "frx_plane_products", soft_ok=False)
    return out, gs


TILES = {"auto": 0, "128x128": 1, "128x256": 2}
TILE_NAMES = {v: k for k, v in TILES.items()}


def set_tile(tile) -> str:
    """Force the slice products' tile configuration ("128x128" or "128x256"); "auto" restores
    the autotuner.  Returns the previous setting's name."""
    code = TILES[tile] if isinstance(tile, str) else int(tile)
    st = _lib.load().frx_set_tile(code)
    if st < 0:
        raise FrxError(st, "frx_set_tile")
    return TILE_NAMES[st]


def last_tile() -> str:
    """Tile configuration of the last slice-product launch made by this host thread."""
    return TILE_NAMES[_lib.load().frx_last_tile()]


def tune_stats(clear: bool = False) -> dict:
    """Autotuner decisions: taken by timing, by the cost model, and cache hits."""
    m, d, h = C.c_longlong(), C.c_longlong(), C.c_longlong()
    _lib.load().frx_tune_stats(C.byref(m), C.byref(d), C.byref(h), 1 if clear else 0)
    return {"measured": m.value, "modelled": d.value, "hits": h.value}


def profile_enable(on: bool = True):
    """Time every slice-product GEMM launch with CUDA events on its stream."""
    _lib.load().frx_profile_enable(1 if on else 0)


def profile_read(reset: bool = False) -> dict:
    p = _lib.Profile()
    st = _lib.load().frx_profile_read(C.byref(p), 1 if reset else 0)
    _check(st, "frx_profile_read", soft_ok=False)
    return p.as_dict()
