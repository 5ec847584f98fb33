"""The replica (weak-scaling) path of bench.py with two CPU ranks over gloo.

Each rank refines its own matrix; the only collectives are the timing barrier and the
max-over-ranks reduction.  Runs without a GPU: the ranks use the CPU oracle on small
matrices in place of the library.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import time

    import bench
    from oracle import refine as orf
    from paper_2602_19090_gb300 import synth
    case = bench.replica_case(rank)
    A, X0, D0, lam = synth.refine_workload(24, 1e2, "spd", case=case)
    bench.barrier(ws)
    t0 = time.perf_counter()
    X, l, info = orf.refine(A, X0, D0, 1e-12, orf.Options())
    ms = (time.perf_counter() - t0) * 1e3 + 10.0 * rank      # ranks differ in time
    ms_max = bench.allmax(ws, ms, device="cpu")
    out[rank] = (case, info["status"], ms, ms_max, bench.job_throughput(ws, 1, ms_max),
                 float(abs(A).sum()))
    dist.destroy_process_group()


def test_two_rank_replicas():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    cases = {r[0] for r in res.values()}
    assert cases == {0, 1}                                  # each rank its own matrix
    assert res[0][5] != res[1][5]
    assert all(r[1] == "converged" for r in res.values())
    ms_max = max(r[2] for r in res.values())
    for r in res.values():
        assert r[3] == pytest.approx(ms_max)                # max over ranks
        assert r[4] == pytest.approx(2 * 1e3 / ms_max)      # whole-job throughput
