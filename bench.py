"""Benchmark: seconds for frx_refine to reach forward error <= 1e-14 at n = 4096 (GB300).

One step = one full refinement (Algorithm 1 iterated with the Sec. 3 / 4.1 rules:
exponent scans, slicing, the three Ozaki products per iteration, residual,
correction, update, stopping test) of a 4096 x 4096 SPD matrix with a geometric
spectrum (cond 1e4, randsvd-like), from a start perturbed by 1e-8, to delta = 1e-14.
Inputs are synthetic and resident in HBM; A alone (134 MB) exceeds the 129 MB L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): every rank refines its own matrix (weak scaling, no collective
on the data path); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("seconds to reach forward error ≤1e-14 at n=4096 vs native-FP64 refinement; "
          "Ozaki GEMM TFLOPS-eq")


def gemm_traffic():
    """DRAM bytes per launch of the tensor-core product kernel from the committed ncu summary,
    or None when the kernel source has changed since those counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "plane_gemm_tc256_n4096_traffic.md")
    src = os.path.join(ROOT, "paper_2602_19090_gb300", "csrc", "gemm_tc.cu")
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        for key in ("traffic_bytes_per_launch:", "kernel_source_sha256_16:"):
            if key in line:
                vals[key] = line.split(key, 1)[1].strip().split()[0]
    if vals.get("kernel_source_sha256_16:") != sha:
        return None
    try:
        return int(vals["traffic_bytes_per_launch:"])
    except (KeyError, ValueError):
        return None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None,
                   help="timed steps (default: 40 for refine and batched, about a second of timed work "
                        "so that the clock sampler sees it; 3 for the other workloads and the reference arm)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=4096)
    p.add_argument("--cond", type=float, default=1e4)
    p.add_argument("--delta", type=float, default=1e-14)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--ref-budget", type=float, default=180.0,
                   help="seconds of oracle refinements the reference arm may spend: it times full "
                        "refinements one after another while the next one still fits, at least one")
    p.add_argument("--no-truth", action="store_true",
                   help="skip the exact-truth companion run that measures the forward error")
    p.add_argument("--no-fp64", action="store_true", help="skip the native-FP64 comparator")
    p.add_argument("--no-gemm", action="store_true", help="skip the stand-alone Ozaki GEMM figures")
    p.add_argument("--workload", choices=["refine", "batched", "configs", "figures", "previous", "gemm", "sparse"],
                   default="refine",
                   help="refine: one n=4096 refinement per step; batched: 256 matrices, n in [32, 512]; "
                        "configs: the n=2048 variants and the n=8192 forward-error sweep; figures: the "
                        "paper's convergence-figure settings with measured forward errors ('previous' is "
                        "an alias); gemm: the ozaki_gemm sweep; sparse: the sparse rule with V over A's nonzeros")
    p.add_argument("--count", type=int, default=256)
    p.add_argument("--sweep-n", default="1024,4096,8192", help="matrix orders of the ozaki_gemm sweep")
    p.add_argument("--tile", default="auto", choices=["auto", "128x128", "128x256"],
                   help="tile configuration of the slice products (auto: the library's autotuner)")
    a = p.parse_args()
    if a.steps is None:
        a.steps = 40 if a.impl == "ours" and a.workload in ("refine", "batched") else 3
    return a


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampling around the timed region; the rows stamped inside it are kept."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 200

    def __init__(self, index):
        self.index = index
        self.t0 = self.t1 = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        # the sampler is running once its first row is out
        t = time.time()
        while self.p is not None and time.time() - t < 5.0 and os.path.getsize(self.f.name) == 0:
            time.sleep(0.02)

    def start(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    @staticmethod
    def _stamp(text):
        import datetime
        try:
            return datetime.datetime.strptime(text.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(1.5 * self.PERIOD_MS / 1e3)     # one more row after the region
        self.p.terminate()
        self.p.wait()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        parsed = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                parsed.append((self._stamp(r[0]), float(r[2]), float(r[3]),
                               {nm for nm, v in zip(names, r[6:10]) if v.strip().lower() == "active"}))
            except (ValueError, IndexError):
                pass
        inside = [q for q in parsed if q[0] is not None and self.t0 is not None and self.t1 is not None
                  and self.t0 <= q[0] <= self.t1]
        where = "inside the timed region"
        if not inside and self.t0 is not None and self.t1 is not None:
            # a region shorter than the sampling period: the rows next to it on either side
            pad = self.PERIOD_MS / 1e3
            inside = [q for q in parsed if q[0] is not None and self.t0 - pad <= q[0] <= self.t1 + pad]
            where = f"within {self.PERIOD_MS} ms of the timed region"
        if not inside:
            inside, where = parsed, "whole sampler run (no timestamps)"
        sm = [q[1] for q in inside]
        reasons = set().union(*[q[3] for q in inside]) if inside else set()
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max((q[2] for q in inside), default=None),
                "reasons": sorted(reasons), "samples": len(sm), "samples_taken": where,
                "region_s": (self.t1 - self.t0) if self.t0 is not None and self.t1 is not None else None}


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, x, device="cuda"):
    """Maximum of a per-rank scalar (the job's time is the slowest rank's)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_case(rank):
    """Each rank refines its own matrix (weak scaling, no data-path collective)."""
    return rank


def job_throughput(ws, units_per_rank, ms_max):
    """Whole-job rate: units all ranks processed / the slowest rank's time."""
    return ws * units_per_rank * 1e3 / ms_max


def cpu_oracle_refine(A, X0, D0, delta):
    """Times one full refinement by the CPU oracle on the host cores, as the oracle stands:
    Algorithm 1 iterated with the Sec. 3 / 4.1 rules and the stopping test, in double-double
    with exact integer slice products.  Returns (cpu_baseline record, refined X, oracle info)."""
    from oracle import refine as orf
    t0 = time.perf_counter()
    X, lam, info = orf.refine(A, X0.copy(), D0.copy(), delta, orf.Options())
    dt = time.perf_counter() - t0
    rec = {"value": dt, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": (f"one full oracle refinement of the workload, timed whole: {info['iters']} iterations, "
                      f"{info['products']} slice products, status {info['status']}; the slice products use "
                      f"numpy's multithreaded FP64 BLAS on all host cores (exact for these integer sums), the "
                      f"rest of the oracle is single-threaded numpy")}
    return rec, X, info


def oracle_warmup(A, X0, D0, delta):
    """A bounded sample of the oracle's work (its plan and the V product on 64 rows): warms
    numpy and the BLAS threads before the timed oracle refinements."""
    from oracle import ozaki as oz
    from oracle import refine as orf
    p = orf.plan(A, X0, D0, delta, orf.Options())
    X1, _ = oz.tau_truncate_cols(X0, p["beta"], p["f"])
    oz.ozaki_product(A[:64], X1, p["kV"], p["sX"], p["kV"] + 1, eL=p["eA"][:64], eR=p["f"])


def truth_companion(api, synth, dev, n, cond, delta, opts):
    """The headline's refinement on an exact-truth matrix of the same order and condition:
    rotated-Hadamard eigenvectors (not FP64 numbers) with a geometric spectrum, start perturbed
    by 1e-8.  Returns the measured forward error ||X - X^||_2 and the run's report."""
    import torch
    A, X0, D0, lam, Qh, Ql, hinfo = synth.rotated_hadamard_workload(n, cond, synth.seed_for(2, 800))
    At = torch.from_numpy(A).to(dev)
    X0t = api.colmajor(torch.from_numpy(X0).to(dev))[0]
    D0t = torch.from_numpy(D0).to(dev)
    Qht, Qlt = torch.from_numpy(Qh).to(dev), torch.from_numpy(Ql).to(dev)
    work = api.workspace(api.refine_workspace_bytes(n, opts), dev)
    _timed_refine(api, At, X0t, D0t, delta, opts, work)
    ms, info, X = _timed_refine(api, At, X0t, D0t, delta, opts, work)
    fe = _forward_error(X, Qht, Qlt)
    fe0 = _forward_error(X0t, Qht, Qlt)
    return {"value": fe["two"], "norm": "2-norm (power iteration), columns sign-aligned", "fro": fe["fro"],
            "max_column": fe["maxcol"], "start": fe0["two"], "delta": delta, "ratio_to_delta": fe["two"] / delta,
            "status": info["status_name"], "iters": info["iters"], "products": info["products"], "ms": ms,
            "workload": (f"exact truth: eigenvectors H R / sqrt(n) (Sylvester Hadamard columns paired by the "
                         f"3-4-5 rotation), n={n}, geometric spectrum cond {cond:g} scaled by 25 "
                         f"(min gap {hinfo['min_gap']:.3g}), start perturbed 1e-8, delta={delta:g}")}


def run_ours(args):
    import numpy as np
    import torch

    from paper_2602_19090_gb300 import api, synth

    ws, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    n, delta = args.n, args.delta
    A, X0, D0, lam = synth.refine_workload(n, args.cond, "spd", case=replica_case(rank))
    At = torch.from_numpy(A).to(dev)
    X0t, _, _ = api.colmajor(torch.from_numpy(X0).to(dev))
    D0t = torch.from_numpy(D0).to(dev)
    X = api.empty_colmajor(n, n, dev)
    D = torch.empty_like(D0t)
    opts = api.Options()
    work = api.workspace(api.refine_workspace_bytes(n, opts), dev)
    api.set_tile(args.tile)

    def one():
        X.copy_(X0t)
        D.copy_(D0t)
        return api.refine(At, X, D, delta, opts, work=work)

    for _ in range(args.warmup):
        info = one()
    torch.cuda.synchronize()
    api.profile_read(reset=True)
    api.profile_enable(True)
    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    clocks.start()
    s.record()
    infos = [one() for _ in range(args.steps)]
    e.record()
    torch.cuda.synchronize()
    clocks.end()
    barrier(ws)
    clk = clocks.stop()
    api.profile_enable(False)
    prof = api.profile_read(reset=True)
    ms = allmax(ws, s.elapsed_time(e)) / args.steps
    info = infos[-1]

    # end to end through the public API with pinned host buffers
    A_h = torch.from_numpy(A).pin_memory()
    X0_h = torch.from_numpy(X0).pin_memory()
    D0_h = torch.from_numpy(D0).pin_memory()
    Xo_h = torch.empty_like(X0_h).pin_memory()
    Do_h = torch.empty_like(D0_h).pin_memory()
    Ad = torch.empty_like(At)
    Xd = torch.empty((n, n), dtype=torch.float64, device=dev)
    Dd = torch.empty_like(D0t)
    torch.cuda.synchronize()
    barrier(ws)
    s2 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    s2.record()
    for _ in range(args.steps):
        Ad.copy_(A_h, non_blocking=True)
        Xd.copy_(X0_h, non_blocking=True)
        Dd.copy_(D0_h, non_blocking=True)
        api.refine(Ad, Xd, Dd, delta, opts, work=work)
        Xo_h.copy_(Xd, non_blocking=True)
        Do_h.copy_(Dd, non_blocking=True)
    e2.record()
    torch.cuda.synchronize()
    e2e_ms = allmax(ws, s2.elapsed_time(e2)) / args.steps

    pk, src = peaks()
    # the GEMM launches run in bursts of a few ms inside a ~30 ms step, far from the
    # seconds-long power-capped loop of the sustained figure: use the burst peak
    peak = pk.get("bf16_tflops")
    achieved = prof["gemm_ops"] / (prof["gemm_ms"] * 1e-3) / 1e12 if prof["gemm_ms"] > 0 else 0.0
    line = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 digit planes, exact int32 plane sums, f64/dd elsewhere",
        "data": "synthetic",
        "config": {"workload": f"refine n={n} SPD geometric cond {args.cond:g}, start perturbed 1e-8, "
                               f"delta={delta:g}", "n": n, "cond": args.cond, "delta": delta,
                   "per_gpu_matrices": 1,
                   "l2": (f"inputs larger than L2 (A alone {A.nbytes / 1e6:.0f} MB > 129 MB)" if A.nbytes > 129e6 else
                          f"A is {A.nbytes / 1e6:.0f} MB, below the 129 MB L2; V's digit planes "
                          f"({info['k_V']} x {4 * n * n / 1e6:.0f} MB) are not"),
                   "parallelism": f"replicas x{ws}"},
        "refine": {"status": info["status_name"], "iters": info["iters"], "err_est": info["err_est"],
                   "step": info["step"], "products": info["products"], "k_V": info["k_V"],
                   "s_X": info["s_X"], "beta": info["beta"]},
        "refinements_per_s": job_throughput(ws, 1, ms),
        "roofline": {"bound": "tensor", "kernel": "slice-product GEMM (digit planes)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if peak else None,
                     # the committed counters were taken on the default workload only
                     "traffic": gemm_traffic() if (n, args.cond, delta) == (4096, 1e4, 1e-14) else None,
                     "peak_source": f"{src} bf16_tflops (burst; sustained {pk.get('bf16_tflops_sustained')})",
                     "gemm_share_of_step": prof["gemm_ms"] / (ms * args.steps) if ms else None},
        "gpu_launches": prof["kernel_launches"],
        "tile": {"used": api.last_tile(), "policy": "autotuned" if args.tile == "auto" else "forced"},
        "e2e": {"value": e2e_ms / 1e3, "unit": "s", "h2d_bytes_per_step": int(A_h.numel() * 8 + X0_h.numel() * 8 + D0_h.numel() * 8),
                "d2h_bytes_per_step": int(Xo_h.numel() * 8 + Do_h.numel() * 8)},
        "clocks": clk,
    }
    if not args.no_fp64:
        # comparator: the same refinement with native FP64 products (cuBLAS DGEMM), timed once
        from paper_2602_19090_gb300 import fp64_refine
        # one untimed run first: the library's FP64 kernels for this size load on first use
        fp64_refine.refine(At, X0t.clone(), D0t, delta)
        Xr = X0t.clone()
        torch.cuda.synchronize()
        s3 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        s3.record()
        Xb, lamb, ib = fp64_refine.refine(At, Xr, D0t, delta)
        e3.record()
        torch.cuda.synchronize()
        b1_ms = allmax(ws, s3.elapsed_time(e3))
        X.copy_(X0t)
        D.copy_(D0t)
        api.refine(At, X, D, delta, opts, work=work)
        diff = (Xb - X).abs().max().item()
        line["fp64_refine"] = {"seconds": b1_ms / 1e3, "status": ib["status"], "iters": ib["iters"],
                               "dgemms": ib["products"], "n_A": ib["nA"], "err_est": ib["err_est"],
                               "speedup_ours_vs_fp64": b1_ms / ms,
                               "max_abs_diff_X_vs_ours": diff,
                               "note": "paper's FP64 slicing (Sec. 4.1 alpha, beta) with cuBLAS DGEMM on the same GPU"}
    if not args.no_gemm:
        # Ozaki GEMM alone (operands N(0,1) * exp(2 N(0,1)), 8 slices per operand): TFLOPS-eq = 2 n^3 / t
        from paper_2602_19090_gb300 import synth as _syn
        Ag = torch.from_numpy(_syn.gemm_operand(n, n, 2.0, 1001)).to(dev)
        Bg = torch.from_numpy(_syn.gemm_operand(n, n, 2.0, 1002)).to(dev)
        Agc, _, _ = api.colmajor(Ag)
        Bgc, _, _ = api.colmajor(Bg)
        ref = (Agc @ Bgc)
        torch.cuda.synchronize()
        s5 = torch.cuda.Event(enable_timing=True)
        e5 = torch.cuda.Event(enable_timing=True)
        s5.record()
        ref = Agc @ Bgc
        e5.record()
        torch.cuda.synchronize()
        dgemm_ms = s5.elapsed_time(e5)
        mag = Agc.abs() @ Bgc.abs()
        gl = {}
        for mode in ("triangular", "full"):
            gw = api.workspace(api._lib.load().frx_ozaki_gemm_workspace_bytes(n, n, n, 8), dev)
            C = api.ozaki_gemm(Agc, Bgc, 8, mode, work=gw)
            torch.cuda.synchronize()
            best = 1e30
            for _ in range(3):
                s4 = torch.cuda.Event(enable_timing=True)
                e4 = torch.cuda.Event(enable_timing=True)
                s4.record()
                C = api.ozaki_gemm(Agc, Bgc, 8, mode, work=gw)
                e4.record()
                torch.cuda.synchronize()
                best = min(best, s4.elapsed_time(e4))
            gl[mode] = {"ms": best, "tflops_eq": 2 * n ** 3 / best / 1e9, "products": 36 if mode == "triangular" else 64,
                        "max_err_vs_dgemm_rel_absAabsB": float(((C - ref).abs() / mag).max())}
            del gw
        line["ozaki_gemm"] = {"n": n, "phi": 2.0, "slices": 8, "dgemm_ms": dgemm_ms,
                              "dgemm_tflops": 2 * n ** 3 / dgemm_ms / 1e9, **gl}
        del Ag, Bg, Agc, Bgc, ref, mag
    if not args.no_truth:
        # the headline workload against a reference X: the native-FP64 comparator iterated to
        # delta = 1e-16 (independent of the frx kernels; checked against the CPU oracle's
        # double-double eigenvectors by a GPU test) ...
        from paper_2602_19090_gb300 import fp64_refine
        T, _, it = fp64_refine.refine(At, X0t, D0t, 1e-16, max_iter=8, xi=0.0)
        X.copy_(X0t)
        D.copy_(D0t)
        ih = api.refine(At, X, D, delta, opts, work=work)
        feh = _forward_error(X, T, torch.zeros_like(T))
        line["forward_error"] = {
            "value": feh["two"], "norm": "2-norm (power iteration), columns sign-aligned", "fro": feh["fro"],
            "delta": delta, "ratio_to_delta": feh["two"] / delta, "status": ih["status_name"],
            "reference": (f"native-FP64 comparator (Sec. 4.1 xi = n) iterated to delta = 1e-16 ({it['status']}, "
                          f"{it['iters']} iterations, est {it['err_est']:.2e})"),
            # ... and an exact-truth matrix of the same order and condition
            "exact_truth_companion": truth_companion(api, synth, dev, n, args.cond, delta, opts)}
        del T
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        cb, Xo, io = cpu_oracle_refine(A, X0, D0, delta)
        X.copy_(X0t)
        D.copy_(D0t)
        ig = api.refine(At, X, D, delta, opts, work=work)
        cb["parity_vs_gpu"] = {"max_abs_diff_X": float(np.max(np.abs(X.cpu().numpy() - Xo))),
                               "iters": [io["iters"], ig["iters"]], "products": [io["products"], ig["products"]],
                               "status": [io["status"], ig["status_name"]]}
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batched(args):
    """Batched workload: `count` matrices, n ~ U{32..512}, cond log-uniform in [1e2, 1e12]."""
    import numpy as np
    import torch

    from paper_2602_19090_gb300 import api, fp64_refine, synth

    ws, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    delta = args.delta if args.delta != 1e-14 else 1e-12
    sizes, conds = synth.batched_sizes(args.count, case=rank)
    probs = []
    for b, (nn, c) in enumerate(zip(sizes, conds)):
        seed = synth.seed_for(3, 1 + b + 1000 * rank)
        A, Q, lam = synth.symmetric_matrix(int(nn), float(c), seed)
        X0, D0 = synth.initial_guess(Q, lam, seed)
        probs.append((A, X0, D0))
    As = [torch.from_numpy(p[0]).to(dev) for p in probs]
    # all starting X (column-major) and D in two flat buffers, so one copy restores every input
    offs = np.concatenate([[0], np.cumsum([p[1].size for p in probs])]).astype(np.int64)
    doffs = np.concatenate([[0], np.cumsum([p[2].size for p in probs])]).astype(np.int64)
    X0flat = torch.from_numpy(np.concatenate([np.asfortranarray(p[1]).ravel(order="F") for p in probs])).to(dev)
    D0flat = torch.from_numpy(np.concatenate([p[2] for p in probs])).to(dev)
    Xflat, Dflat = X0flat.clone(), D0flat.clone()
    Xs = [Xflat[offs[b]:offs[b + 1]].view(int(p[1].shape[1]), int(p[1].shape[0])).t() for b, p in enumerate(probs)]
    Ds = [Dflat[doffs[b]:doffs[b + 1]] for b in range(len(probs))]
    X0s = [X0flat[offs[b]:offs[b + 1]].view(int(p[1].shape[1]), int(p[1].shape[0])).t() for b, p in enumerate(probs)]
    D0s = [D0flat[doffs[b]:doffs[b + 1]] for b in range(len(probs))]
    lib = api._lib.load()
    import ctypes as C
    o = api.Options().to_c()
    nn = (C.c_int64 * len(As))(*[a.shape[0] for a in As])
    work = api.workspace(lib.frx_refine_batched_workspace_bytes(nn, len(As), C.byref(o)), dev)

    def one():
        Xflat.copy_(X0flat)
        Dflat.copy_(D0flat)
        return api.refine_batched(As, Xs, Ds, delta, work=work)

    api.set_tile(args.tile)

    for _ in range(args.warmup):
        infos = one()
    api.profile_read(reset=True)
    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    clocks.start()
    s.record()
    for _ in range(args.steps):
        infos = one()
    e.record()
    torch.cuda.synchronize()
    clocks.end()
    barrier(ws)
    clk = clocks.stop()
    prof = api.profile_read(reset=True)
    ms = allmax(ws, s.elapsed_time(e)) / args.steps
    stats = {}
    for i in infos:
        stats[i["status_name"]] = stats.get(i["status_name"], 0) + 1
    # algorithmic work of the batch's slice products: every product of matrix b is an n_b x n_b x
    # n_b digit-plane GEMM (2 n_b^3 operations); its rate over the whole step is a lower bound on
    # the grouped tensor-core launches' own rate (which the step shares with everything else)
    gemm_ops = float(sum(int(i["products"]) * 2.0 * float(p[0].shape[0]) ** 3 for i, p in zip(infos, probs)))
    pk, src = peaks()
    peak = pk.get("bf16_tflops")
    step_rate = gemm_ops / (ms * 1e-3) / 1e12
    slice_work = {"tflop_per_step": gemm_ops / 1e12, "tflops_over_whole_step": step_rate,
                  "peak": peak, "peak_source": src,
                  "fraction_of_peak_over_whole_step": step_rate / peak if peak else None,
                  "note": "lower bound on the grouped slice-product launches' rate: the step also holds the "
                          "element-wise, slicing and plan stages"}

    # end to end through the public API: every step copies all matrices, starting vectors and
    # estimates in from pinned host memory and the refined X, D back
    aoffs = np.concatenate([[0], np.cumsum([p[0].size for p in probs])]).astype(np.int64)
    A_h = torch.from_numpy(np.concatenate([p[0].ravel() for p in probs])).pin_memory()
    X0_h = X0flat.cpu().pin_memory()
    D0_h = D0flat.cpu().pin_memory()
    Xo_h = torch.empty_like(X0_h).pin_memory()
    Do_h = torch.empty_like(D0_h).pin_memory()
    Aflat = torch.empty(A_h.shape, dtype=torch.float64, device=dev)
    Aviews = [Aflat[aoffs[b]:aoffs[b + 1]].view(int(p[0].shape[0]), int(p[0].shape[1])) for b, p in enumerate(probs)]

    def one_e2e():
        Aflat.copy_(A_h, non_blocking=True)
        Xflat.copy_(X0_h, non_blocking=True)
        Dflat.copy_(D0_h, non_blocking=True)
        out = api.refine_batched(Aviews, Xs, Ds, delta, work=work)
        Xo_h.copy_(Xflat, non_blocking=True)
        Do_h.copy_(Dflat, non_blocking=True)
        return out

    one_e2e()        # untimed: these buffers get their own launch plan
    torch.cuda.synchronize()
    barrier(ws)
    s2 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    s2.record()
    for _ in range(args.steps):
        one_e2e()
    e2.record()
    torch.cuda.synchronize()
    e2e_ms = allmax(ws, s2.elapsed_time(e2)) / args.steps
    e2e = {"value": job_throughput(ws, args.count, e2e_ms), "unit": "matrices/s",
           "h2d_bytes_per_step": int((A_h.numel() + X0_h.numel() + D0_h.numel()) * 8),
           "d2h_bytes_per_step": int((Xo_h.numel() + Do_h.numel()) * 8)}
    del Aflat, Aviews

    # per-matrix native-FP64 loop (cuBLAS DGEMM), once
    fstats, fp64_ms = {}, None
    if not args.no_fp64:
        # one untimed pass first: cuBLAS loads its FP64 kernels for each new shape on first use
        for A, x0, d0 in zip(As, X0s, D0s):
            fp64_refine.refine(A, x0.clone(), d0.clone(), delta)
        torch.cuda.synchronize()
        s2 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        s2.record()
        for A, x0, d0 in zip(As, X0s, D0s):
            _, _, ib = fp64_refine.refine(A, x0.clone(), d0.clone(), delta)
            fstats[ib["status"]] = fstats.get(ib["status"], 0) + 1
        e2.record()
        torch.cuda.synchronize()
        fp64_ms = s2.elapsed_time(e2)
    line = {
        "metric": "matrices/s refined to the forward-error target (batched)",
        "value": job_throughput(ws, args.count, ms),
        "unit": "matrices/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 digit planes, exact int32 plane sums, f64/dd elsewhere", "data": "synthetic",
        "config": {"workload": f"batched: {args.count} matrices, n ~ U[32, 512], cond log-uniform [1e2, 1e12], "
                               f"start perturbed 1e-8, delta={delta:g}", "count": args.count,
                   "n_min": int(sizes.min()), "n_max": int(sizes.max()), "delta": delta,
                   "l2": (f"inputs larger than L2 (A, X and D of the batch: "
                          f"{(sum(p[0].nbytes + p[1].nbytes + p[2].nbytes for p in probs)) / 1e6:.0f} MB > 129 MB)")},
        "statuses": stats, "gpu_launches": prof["kernel_launches"],
        "slice_product_work": slice_work,
        "e2e": e2e,
        "tile": {"used": api.last_tile(), "policy": "autotuned" if args.tile == "auto" else "forced",
                 "tuner": api.tune_stats()},
        "fp64_loop": ({"seconds": fp64_ms / 1e3, "matrices_per_s": args.count * 1e3 / fp64_ms, "statuses": fstats,
                       "speedup_ours": fp64_ms / ms} if fp64_ms else None),
        "clocks": clk,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_batched(probs, delta)
    if rank == 0:
        print(json.dumps(line), flush=True)


def cpu_oracle_batched(probs, delta, budget_s=15.0):
    """The CPU oracle's full refinement of the batch's matrices in order, until about
    `budget_s` seconds have passed (at least one matrix): matrices/s over that sample."""
    from oracle import refine as orf
    t0 = time.perf_counter()
    done, sizes = 0, []
    for A, X0, D0 in probs:
        orf.refine(A, X0, D0, delta, orf.Options())
        done += 1
        sizes.append(int(A.shape[0]))
        if time.perf_counter() - t0 > budget_s:
            break
    t = time.perf_counter() - t0
    return {"value": done / t, "unit": "matrices/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"full oracle refinement of the batch's first {done} matrices (n = {sizes}) took "
                       f"{t:.1f} s; the slice products use numpy's multithreaded FP64 BLAS, the rest is "
                       f"single-threaded numpy")}


def _timed_refine(api, A, X0, D0, delta, opts, work, reps=1):
    import torch
    best, info, X = 1e30, None, None
    for _ in range(reps):
        X = X0.clone()
        D = D0.clone()
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        info = api.refine(A, X, D, delta, opts, work=work)
        e.record()
        torch.cuda.synchronize()
        best = min(best, s.elapsed_time(e))
    return best, info, X


def _timed_fp64(At, X0t, D0t, delta):
    import torch

    from paper_2602_19090_gb300 import fp64_refine
    torch.cuda.synchronize()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record()
    Xb, _, ib = fp64_refine.refine(At, X0t.clone(), D0t.clone(), delta)
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e), ib, Xb


def _forward_error(X, Qh, Ql):
    """||X - Q||_2 with columns sign-aligned (Q = Qh + Ql known exactly); also the Frobenius
    norm and the largest column norm, which bracket it.  The 2-norm is a 40-step power
    iteration on the difference scaled to unit Frobenius norm, in single precision."""
    import torch
    sg = torch.sign((Qh * X).sum(0))
    sg[sg == 0] = 1
    D = (X * sg - Qh) - Ql
    fro = float(torch.linalg.norm(D))
    col = float(torch.linalg.norm(D, dim=0).max())
    if fro == 0.0:
        return {"two": 0.0, "fro": 0.0, "maxcol": 0.0}
    Ds = (D / fro).float()
    g = torch.Generator(device=D.device).manual_seed(7)
    v = torch.randn(D.shape[1], device=D.device, generator=g)
    v /= torch.linalg.norm(v)
    lam2 = 0.0
    for _ in range(40):
        w = Ds.T @ (Ds @ v)
        lam2 = float(torch.linalg.norm(w))
        v = w / lam2
    return {"two": math.sqrt(lam2) * fro, "fro": fro, "maxcol": col}


def run_configs(args):
    """Refinement configurations beside the headline one (one JSON line):
    the n=2048 variants of the randsvd-like workload with native-FP64 times, the n=8192
    cond-1e12 target sweep, and exact-truth workloads (Hadamard eigenvectors) with the
    forward error of both paths measured against the known eigenvectors."""
    import torch

    from paper_2602_19090_gb300 import api, synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    out = {"metric": "configs", "variants_n2048": [], "sweep_n8192": [], "exact_truth_n4096": [],
           "exact_truth_sweep_n8192": []}

    def dev_inputs(A, X0, D0):
        return (torch.from_numpy(A).to(dev), api.colmajor(torch.from_numpy(X0).to(dev))[0],
                torch.from_numpy(D0).to(dev))

    # warm the native-FP64 path (library handles, kernels) on a small problem
    A, X0, D0, _ = synth.refine_workload(256, 1e4, "spd", case=99)
    _timed_fp64(*dev_inputs(A, X0, D0), 1e-12)

    n = 2048
    work = api.workspace(api.refine_workspace_bytes(n), dev)
    for cond, variant in ((1e4, "spd"), (1e10, "spd"), (1e14, "spd"), (1e4, "indefinite"), (1e4, "clustered")):
        A, X0, D0, lam = synth.refine_workload(n, cond, variant, case=int(cond) % 97 + len(variant))
        At, X0t, D0t = dev_inputs(A, X0, D0)
        opts = api.Options(cluster_omega=-1.0 if variant == "clustered" else 0.0)
        for delta in (1e-10, 1e-14):
            ms, info, X = _timed_refine(api, At, X0t, D0t, delta, opts, work, reps=2)
            rec = {"cond": cond, "variant": variant, "delta": delta, "ms": ms, "status": info["status_name"],
                   "iters": info["iters"], "products": info["products"], "k_V": info["k_V"], "s_X": info["s_X"],
                   "err_est": info["err_est"], "clustered_pairs": info["clustered_pairs"]}
            fms, ib, Xb = _timed_fp64(At, X0t, D0t, delta)
            rec.update(fp64_ms=fms, fp64_status=ib["status"], fp64_iters=ib["iters"],
                       max_abs_diff_vs_fp64=float((Xb - X).abs().max()))
            out["variants_n2048"].append(rec)
            print(json.dumps(rec), file=sys.stderr, flush=True)
            if not args.no_cpu_baseline and cond == 1e4 and variant == "spd" and delta == 1e-14:
                # the CPU oracle beside the n = 2048 refinement, on the headline's sampled V product
                out["cpu_baseline_n2048"] = cpu_oracle_refine(A, X0, D0, delta)[0]
        del At, X0t, D0t
    del work

    # exact truth, n = 4096 (the geometric spectra are kept exactly for cond 1e4 and 1e10)
    n = 4096
    work = api.workspace(api.refine_workspace_bytes(n), dev)
    for cond, variant in ((1e4, "spd"), (1e10, "spd"), (1e4, "indefinite"), (1e10, "indefinite")):
        A, X0, D0, lam, Qh, Ql, hinfo = synth.hadamard_workload(n, cond, synth.seed_for(2, 500), variant=variant)
        At, X0t, D0t = dev_inputs(A, X0, D0)
        Qht, Qlt = torch.from_numpy(Qh).to(dev), torch.from_numpy(Ql).to(dev)
        for delta in (1e-10, 1e-14):
            ms, info, X = _timed_refine(api, At, X0t, D0t, delta, api.Options(), work, reps=2)
            fe = _forward_error(X, Qht, Qlt)
            fms, ib, Xb = _timed_fp64(At, X0t, D0t, delta)
            fe_b = _forward_error(Xb, Qht, Qlt)
            rec = {"cond": cond, "variant": variant, "delta": delta, "min_gap": hinfo["min_gap"], "ms": ms,
                   "status": info["status_name"], "iters": info["iters"], "products": info["products"],
                   "k_V": info["k_V"], "s_X": info["s_X"], "err_est": info["err_est"], "forward_error": fe,
                   "fp64_ms": fms, "fp64_status": ib["status"], "fp64_iters": ib["iters"], "fp64_forward_error": fe_b}
            out["exact_truth_n4096"].append(rec)
            print(json.dumps(rec), file=sys.stderr, flush=True)
        del At, X0t, D0t, Qht, Qlt
    del work

    # n = 8192, cond 1e12: the randsvd-like workload (no reference eigenvectors: the estimate
    # and the distance to the native-FP64 result are reported) ...
    n = 8192
    A, X0, D0, lam = synth.refine_workload(n, 1e12, "spd", case=4)
    At, X0t, D0t = dev_inputs(A, X0, D0)
    del A, X0
    work = api.workspace(api.refine_workspace_bytes(n), dev)
    for k in range(8, 16):
        delta = 10.0 ** (-k)
        ms, info, X = _timed_refine(api, At, X0t, D0t, delta, api.Options(), work)
        rec = {"delta": delta, "ms": ms, "status": info["status_name"], "iters": info["iters"],
               "products": info["products"], "k_V": info["k_V"], "k_W": info["k_W"], "k_U": info["k_U"],
               "s_X": info["s_X"], "beta": info["beta"], "err_est": info["err_est"], "step": info["step"]}
        if k in (8, 12):
            fms, ib, Xb = _timed_fp64(At, X0t, D0t, delta)
            rec.update(fp64_ms=fms, fp64_status=ib["status"], fp64_iters=ib["iters"],
                       max_abs_diff_vs_fp64=float((Xb - X).abs().max()))
        out["sweep_n8192"].append(rec)
        print(json.dumps(rec), file=sys.stderr, flush=True)
    del At, X0t, D0t
    # ... and its exact-truth analog (Hadamard eigenvectors, geometric magnitudes with the
    # smallest ones raised to distinct integers), where both forward errors are measured
    A, X0, D0, lam, Qh, Ql, hinfo = synth.hadamard_workload(n, 1e12, synth.seed_for(4, 500))
    At, X0t, D0t = dev_inputs(A, X0, D0)
    Qht, Qlt = torch.from_numpy(Qh).to(dev), torch.from_numpy(Ql).to(dev)
    del A, X0, Qh, Ql
    for k in range(8, 16):
        delta = 10.0 ** (-k)
        ms, info, X = _timed_refine(api, At, X0t, D0t, delta, api.Options(), work)
        rec = {"delta": delta, "min_gap": hinfo["min_gap"], "ms": ms, "status": info["status_name"],
               "iters": info["iters"], "products": info["products"], "k_V": info["k_V"], "k_W": info["k_W"],
               "k_U": info["k_U"], "s_X": info["s_X"], "beta": info["beta"], "err_est": info["err_est"],
               "forward_error": _forward_error(X, Qht, Qlt)}
        if k in (8, 12):
            fms, ib, Xb = _timed_fp64(At, X0t, D0t, delta)
            rec.update(fp64_ms=fms, fp64_status=ib["status"], fp64_iters=ib["iters"],
                       fp64_forward_error=_forward_error(Xb, Qht, Qlt))
        out["exact_truth_sweep_n8192"].append(rec)
        print(json.dumps(rec), file=sys.stderr, flush=True)
    print(json.dumps(out), flush=True)


def run_figures(args):
    """The settings of the paper's convergence figures (Sec. 4.2: randsvd-like matrices, cond 1e10,
    n = 1024/4096/8192, delta = 1e-8/1e-10/1e-12), four arms each:
      default      eq. proposed_beta with xi = 1 (the library's default);
      sec41        the "n delta" form of the Sec. 4.1 experiments (xi = n);
      previous     X kept at full FP64 width (7 digit planes), no truncation rule: the GB300 form
                   of the earlier method that slices both operands;
      fp64         the native-FP64 comparator (cuBLAS DGEMM, the paper's FP64 slicing), xi = 1.
    Each arm: status, iterations, slice products, time and the measured forward error
    ||X - X^||_2 against a reference X: the native-FP64 comparator in its Sec. 4.1 form (xi = n)
    iterated to delta = 1e-16 (an
    implementation independent of the frx kernels; its agreement with the CPU oracle's
    double-double eigenvectors is a GPU test).  Then the exact-truth rotated-Hadamard matrix
    (n = 4096, cond 1e10), whose eigenvectors are known exactly."""
    import torch

    from paper_2602_19090_gb300 import api, fp64_refine, synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    out = {"metric": "figure_settings", "randsvd_cond1e10": [], "exact_truth_rotated_n4096_cond1e10": []}
    arms = (("default", api.Options()), ("sec41", api.Options(xi=0.0)), ("previous", api.Options(x_planes=7)))

    def dev_inputs(A, X0, D0):
        return (torch.from_numpy(A).to(dev), api.colmajor(torch.from_numpy(X0).to(dev))[0],
                torch.from_numpy(D0).to(dev))

    def arm_record(ms, info, X, ref, refl=None):
        return {"ms": ms, "status": info["status_name"], "iters": info["iters"], "products": info["products"],
                "k_V": info["k_V"], "s_X": info["s_X"], "err_est": info["err_est"],
                "forward_error": _forward_error(X, ref, refl if refl is not None else torch.zeros_like(ref))["two"]}

    sizes = [int(x) for x in args.sweep_n.split(",")]
    for n in sizes:
        A, X0, D0, lam = synth.refine_workload(n, 1e10, "spd", case=600 + n % 97)
        At, X0t, D0t = dev_inputs(A, X0, D0)
        del A, X0
        T, _, it = fp64_refine.refine(At, X0t, D0t, 1e-16, max_iter=8, xi=0.0)
        work = api.workspace(api.refine_workspace_bytes(n), dev)
        for delta in (1e-8, 1e-10, 1e-12):
            rec = {"n": n, "delta": delta, "reference": {"status": it["status"], "iters": it["iters"],
                                                        "err_est": it["err_est"]}}
            for name, opts in arms:
                ms, info, X = _timed_refine(api, At, X0t, D0t, delta, opts, work, reps=2)
                rec[name] = arm_record(ms, info, X, T)
            fms, ib, Xb = _timed_fp64(At, X0t, D0t, delta)
            rec["fp64"] = {"ms": fms, "status": ib["status"], "iters": ib["iters"], "dgemms": ib["products"],
                           "forward_error": _forward_error(Xb, T, torch.zeros_like(T))["two"]}
            out["randsvd_cond1e10"].append(rec)
            print(json.dumps(rec), file=sys.stderr, flush=True)
        del At, X0t, D0t, T, work
        torch.cuda.empty_cache()
    n = 4096
    A, X0, D0, lam, Qh, Ql, hinfo = synth.rotated_hadamard_workload(n, 1e10, synth.seed_for(2, 700))
    At, X0t, D0t = dev_inputs(A, X0, D0)
    Qht, Qlt = torch.from_numpy(Qh).to(dev), torch.from_numpy(Ql).to(dev)
    work = api.workspace(api.refine_workspace_bytes(n), dev)
    for delta in (1e-8, 1e-10, 1e-12):
        rec = {"n": n, "delta": delta, "min_gap": hinfo["min_gap"]}
        for name, opts in arms:
            ms, info, X = _timed_refine(api, At, X0t, D0t, delta, opts, work, reps=2)
            rec[name] = arm_record(ms, info, X, Qht, Qlt)
        out["exact_truth_rotated_n4096_cond1e10"].append(rec)
        print(json.dumps(rec), file=sys.stderr, flush=True)
    print(json.dumps(out), flush=True)


def run_sparse(args):
    """The sparse-matrix setting of Sec. 4 (sparse_rule): stand-ins for the paper's ELSES and
    SuiteSparse matrices (not in the container) - a band matrix (k = 5 nonzeros per row) and
    symmetric matrices with about 8 and 16 nonzeros per row at random positions, n = 4096,
    delta = 1e-12. Each is refined with V = A X^(1) over A's nonzeros (FRX_SPARSE_V=1), with the
    dense tensor-core V product (FRX_SPARSE_V=0) - identical bits required - and with the
    library's automatic choice (sparse when nnz * 160 <= n); CUDA-event times, best of 3."""
    import numpy as np
    import torch

    from paper_2602_19090_gb300 import api, synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    out = {"metric": "sparse_rule", "cases": []}
    n, delta = args.n, 1e-12
    work = api.workspace(api.refine_workspace_bytes(n), dev)
    cases = (("band, k = 5", lambda: synth.banded_workload(n, 2, 31)),
             ("random pattern, ~8 per row", lambda: synth.random_sparse_workload(n, 8, 33)),
             ("random pattern, ~16 per row", lambda: synth.random_sparse_workload(n, 16, 32)))
    for name, make in cases:
        A, X0, D0, lam = make()
        At = torch.from_numpy(A).to(dev)
        X0t = api.colmajor(torch.from_numpy(X0).to(dev))[0]
        D0t = torch.from_numpy(D0).to(dev)
        nnz = int(np.max(np.count_nonzero(A, axis=1)))
        rec = {"case": name, "n": n, "max_row_nonzeros": nnz, "delta": delta,
               "auto_choice": "sparse" if nnz * 160 <= n else "dense"}
        Xs = {}
        for flag, key in (("1", "sparse_v"), ("0", "dense_v"), (None, "auto")):
            if flag is None:
                os.environ.pop("FRX_SPARSE_V", None)
            else:
                os.environ["FRX_SPARSE_V"] = flag
            ms, info, X = _timed_refine(api, At, X0t, D0t, delta, api.Options(sparse_rule=True), work, reps=3)
            Xs[key] = X
            rec[key] = {"ms": ms, "status": info["status_name"], "iters": info["iters"], "products": info["products"],
                        "k_V": info["k_V"], "s_X": info["s_X"], "err_est": info["err_est"]}
        os.environ.pop("FRX_SPARSE_V", None)
        rec["identical_X"] = bool(torch.equal(Xs["sparse_v"], Xs["dense_v"]) and torch.equal(Xs["auto"], Xs["dense_v"]))
        rec["speedup_sparse_over_dense"] = rec["dense_v"]["ms"] / rec["sparse_v"]["ms"]
        out["cases"].append(rec)
        print(json.dumps(rec), file=sys.stderr, flush=True)
        del At, X0t, D0t, Xs
    print(json.dumps(out), flush=True)


def run_gemm_sweep(args):
    """ozaki_gemm over n = 1024/4096/8192, phi = 0.5/2/4, k = 4/8/12/16 planes, both product
    sets: time (CUDA events, best of 3), TFLOPS-eq = 2 n^3 / time, the slice-product kernel's own
    rate, and the error against the same product at 16 planes with all pairs (128 bits of each
    operand), relative to |A||B|; a DGEMM's error on the same scale is given for context."""
    import torch

    from paper_2602_19090_gb300 import api, synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    api.set_tile(args.tile)
    out = {"metric": "ozaki_gemm_sweep", "cases": []}
    sizes = tuple(int(v) for v in args.sweep_n.split(","))
    for n in sizes:
        for phi in (0.5, 2.0, 4.0):
            # column-major operands, so that the timed calls do no layout copies
            A = api.colmajor(torch.from_numpy(synth.gemm_operand(n, n, phi, synth.seed_for(1, 10 + int(phi * 2)))).to(dev))[0]
            B = api.colmajor(torch.from_numpy(synth.gemm_operand(n, n, phi, synth.seed_for(1, 20 + int(phi * 2)))).to(dev))[0]
            work = api.workspace(api.ozaki_gemm_workspace_bytes(n, n, n, 16), dev)
            Rh, Rl = api.ozaki_gemm(A, B, 16, "full", return_lo=True, work=work)
            mag = torch.abs(A) @ torch.abs(B)
            mag = torch.where(mag > 0, mag, torch.ones_like(mag))
            D = A @ B
            dgemm_err = float((((D - Rh) - Rl).abs() / mag).max())
            for k in (4, 8, 12, 16):
                for mode in ("triangular", "full"):
                    C = api.ozaki_gemm(A, B, k, mode, work=work)
                    torch.cuda.synchronize()
                    best = 1e30
                    api.profile_read(reset=True)
                    api.profile_enable(True)
                    for _ in range(3):
                        s0 = torch.cuda.Event(enable_timing=True)
                        e0 = torch.cuda.Event(enable_timing=True)
                        s0.record()
                        C = api.ozaki_gemm(A, B, k, mode, work=work)
                        e0.record()
                        torch.cuda.synchronize()
                        best = min(best, s0.elapsed_time(e0))
                    api.profile_enable(False)
                    pr = api.profile_read(reset=True)
                    products = k * (k + 1) // 2 if mode == "triangular" else k * k
                    err = float((((C - Rh) - Rl).abs() / mag).max())
                    rec = {"n": n, "phi": phi, "k": k, "mode": mode, "products": products, "ms": best,
                           "tflops_eq": 2.0 * n ** 3 / (best * 1e-3) / 1e12,
                           "gemm_kernel_tflops": pr["gemm_ops"] / (pr["gemm_ms"] * 1e-3) / 1e12 if pr["gemm_ms"] else None,
                           "gemm_share": pr["gemm_ms"] / 3 / best if pr["gemm_ms"] else None,
                           "tile": api.last_tile(),
                           "max_err_rel_absAabsB": err, "dgemm_err_rel_absAabsB": dgemm_err}
                    out["cases"].append(rec)
                    print(json.dumps(rec), file=sys.stderr, flush=True)
            del A, B, work, Rh, Rl, mag, D
    if not args.no_cpu_baseline:
        # the CPU oracle's ozaki_gemm on one case of the sweep (n = 1024, phi = 2, 8 planes)
        from oracle import ozaki as oz
        n = 1024
        A = synth.gemm_operand(n, n, 2.0, synth.seed_for(1, 14))
        B = synth.gemm_operand(n, n, 2.0, synth.seed_for(1, 24))
        base = {}
        for mode in ("triangular", "full"):
            t0 = time.perf_counter()
            oz.ozaki_gemm(A, B, 8, mode)
            t = time.perf_counter() - t0
            base[mode] = {"seconds": t, "tflops_eq": 2.0 * n ** 3 / t / 1e12}
        out["cpu_baseline"] = {"value": base["triangular"]["tflops_eq"], "unit": "TFLOPS-eq", "cores": os.cpu_count(),
                               "kind": "oracle", "per_mode": base,
                               "sample": "oracle ozaki_gemm, n = 1024, phi = 2, 8 planes per operand (the slice "
                                         "products use numpy's multithreaded FP64 BLAS, exact for these sums)"}
    print(json.dumps(out), flush=True)


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, timed on the host cores on this arm's
    workload.  Each step is one full oracle refinement; warm-up steps are a bounded sample
    (the oracle's plan and V product on 64 rows).  Full refinements are timed one after another
    while the next still fits in --ref-budget seconds (at least one); `steps` reports how many
    ran, so that steps x ms_per_step is the time actually spent."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2602_19090_gb300 import synth
    n, delta = args.n, args.delta
    A, X0, D0, lam = synth.refine_workload(n, args.cond, "spd", case=0)
    for _ in range(args.warmup):
        oracle_warmup(A, X0, D0, delta)
    recs = []
    t_start = time.perf_counter()
    for _ in range(max(args.steps, 1)):
        rec, _, _ = cpu_oracle_refine(A, X0, D0, delta)
        recs.append(rec)
        if time.perf_counter() - t_start + rec["value"] > args.ref_budget:
            break
    value = statistics.mean([r["value"] for r in recs])
    cb = dict(recs[-1])
    cb["value"] = value
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": 1,
        "steps": len(recs), "requested_steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3,
        "step_values_s": [r["value"] for r in recs],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int64/f64/dd",
        "data": "synthetic",
        "config": {"workload": f"refine n={n} SPD geometric cond {args.cond:g}, start perturbed 1e-8, "
                               f"delta={delta:g}", "n": n},
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "configs":
        run_configs(args)
    elif args.workload in ("figures", "previous"):
        run_figures(args)
    elif args.workload == "gemm":
        run_gemm_sweep(args)
    elif args.workload == "sparse":
        run_sparse(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
