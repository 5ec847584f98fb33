"""The update's roundings of X1 + U (Alg. 1's update, one rounding), checked on the host.

`tests/host_rounding_check.cu` compiles the library's rounding helpers as host code (nvcc, no GPU
needed) and runs them on random, tie and binade-edge inputs, with x1 also next to the subnormal
range and x1 = 0.  Where the on-grid form and the exact 128-bit form both succeed their bits
must agree, and every result either form returns must equal the correctly rounded value of
x1 + N 2^c computed with Python's exact rationals (float(Fraction) rounds to nearest, ties to
even, subnormals included): a form that cannot give that value in the normal range has to
decline, and the kernel then takes its general path.
"""
import os
import shutil
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bits_to_float(u):
    import struct
    return struct.unpack("<d", struct.pack("<Q", u))[0]


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("hostround") / "host_rounding_check"
    cmd = [nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(ROOT, "paper_2602_19090_gb300", "csrc"),
           os.path.join(ROOT, "tests", "host_rounding_check.cu"), "-o", str(out)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(out)


def test_on_grid_rounding_matches_exact_path_and_rationals(checker, tmp_path):
    dump = tmp_path / "grid_cases.txt"
    r = subprocess.run([checker, "2000000", "20261204", str(dump), "40000"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    fields = dict(zip(r.stdout.split()[0::2], map(int, r.stdout.split()[1::2])))
    assert fields["mismatches"] == 0
    assert fields["both"] > 100000 and fields["ties"] > 100000      # both paths and exact ties exercised
    assert fields["tiny"] > 100000
    checked = {"G": 0, "E": 0}
    near_bottom = 0
    for line in dump.read_text().split("\n"):
        if not line:
            continue
        form, xb, c, hi, lo, rb = line.split()
        x1 = _bits_to_float(int(xb, 16))
        N = (int(hi, 16) << 64) | int(lo, 16)
        if N >= 1 << 127:
            N -= 1 << 128
        exact = Fraction(x1) + Fraction(N) * Fraction(2) ** int(c)
        got = _bits_to_float(int(rb, 16))
        assert float(exact) == got, line
        if exact != 0 and abs(exact) < Fraction(2) ** -990:
            near_bottom += 1
        checked[form] += 1
    assert checked["G"] == fields["dumped"] and checked["G"] >= 20000
    assert checked["E"] == fields["dumped_e"] and checked["E"] >= 20000
    assert near_bottom > 1000                                       # results close to 2^-1022
