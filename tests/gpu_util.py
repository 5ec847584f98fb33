"""Helpers for GPU tests (imported only by tests marked gpu)."""
import numpy as np
import torch


def dev():
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def bf16_digits(planes):
    """uint16 bf16 bit patterns (stored as int16) -> int64 digits."""
    p = planes.cpu().numpy().astype(np.uint16).astype(np.uint32) << 16
    return p.view(np.float32).astype(np.int64)


def group_sums(S, kL, kR, T, gs):
    """Combine per-anti-diagonal integer sums into the int64 groups the library returns."""
    tmax = min(T, kL + kR)
    groups = []
    t0 = 2
    while t0 <= tmax:
        t1 = min(t0 + gs - 1, tmax)
        acc = None
        for t in range(t0, t1 + 1):
            St = S.get(t)
            St = St.astype(object) if St is not None else 0
            acc = St if acc is None else acc * 256 + St     # 8-bit digits: planes 2^8 apart
        groups.append(acc)
        t0 = t1 + 1
    return groups
