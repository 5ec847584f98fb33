"""Writes tests/golden/workload0_oracle.json from the CPU oracle only.

Workload: n = 64, cond 1e8 SPD (geometric spectrum), start perturbed by 1e-8,
delta = 1e-14 (the small refinement case).  Stored: per-iteration plan numbers
(beta, alpha, s_X, k_V, k_W, k_U, products) of the Sec. 4.1 rule and the forward
error against the double-double reference eigenvectors.  Run from the repo root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import refine as rf, truth as tr  # noqa: E402
from paper_2602_19090_gb300 import synth  # noqa: E402


def main():
    A, X0, D0 = synth.workload0()
    Xh, Xl, _, _ = tr.eigvecs_dd(A, X0)
    out = {}
    for name, opts in (("auto", rf.Options()), ("fixed8", rf.Options(slices_A=8, max_iter=3))):
        hist = []
        _, _, info = rf.refine(A, X0, D0, 1e-14, opts, history=hist)
        out[name] = dict(status=info["status"], iters=info["iters"], products=info["products"],
                         steps=[dict(beta=h["beta"], alpha=h["alpha"], sX=h["sX"], kV=h["kV"],
                                     kW=h["kW"], kU=h["kU"], products=h["products"],
                                     forward_error=tr.forward_error(Xh, Xl, h["X"]))
                                for h in hist])
    out["initial_forward_error"] = tr.forward_error(Xh, Xl, X0)
    path = os.path.join(ROOT, "tests", "golden", "workload0_oracle.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(path)


if __name__ == "__main__":
    main()
