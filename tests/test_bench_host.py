"""Host-side logic of bench.py that needs no GPU: the clock record kept from the timed region,
the timed oracle refinement, the reference arm's step accounting, the per-workload step
defaults, the ncu traffic figure's tie to the profiled kernel source and the whole-job rate."""
import datetime
import sys
import time

import pytest


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def _stamp(t):
    return datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]


def _fake_clocks(bench, tmp_path, rows, t0, t1):
    # rows: (seconds after t0, SM MHz, sw_power_cap active?)
    path = tmp_path / "clocks.csv"
    with open(path, "w") as f:
        for dt, mhz, cap in rows:
            f.write(f"{_stamp(t0 + dt)}, 0, {mhz}, 2070, 900.00 W, 0x0, Not Active, Not Active, "
                    f"Not Active, {'Active' if cap else 'Not Active'}\n")
    c = bench.Clocks.__new__(bench.Clocks)
    c.f = open(path)
    c.p = type("P", (), {"terminate": lambda s: None, "wait": lambda s: None})()
    c.t0, c.t1 = t0, t1
    c.PERIOD_MS = 200
    return c


def test_clocks_keep_only_the_timed_region(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(time, "sleep", lambda s: None)
    t0 = time.time()
    c = _fake_clocks(bench, tmp_path, [(-0.4, 1100, False), (0.1, 2070, False), (0.3, 2050, True),
                                       (0.5, 2070, False), (0.9, 900, False)], t0, t0 + 0.6)
    rec = c.stop()
    assert rec["samples"] == 3 and rec["samples_taken"] == "inside the timed region"
    assert rec["sm_mhz"] == 2070 and rec["sm_max_mhz"] == 2070
    assert rec["reasons"] == ["sw_power_cap"]


def test_clocks_short_region_takes_the_adjacent_rows(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(time, "sleep", lambda s: None)
    t0 = time.time()
    c = _fake_clocks(bench, tmp_path, [(-0.15, 2040, False), (0.12, 2060, False), (0.6, 800, False)],
                     t0, t0 + 0.05)
    rec = c.stop()
    assert rec["samples"] == 2 and rec["samples_taken"].startswith("within 200 ms")
    assert rec["sm_mhz"] == 2050 and rec["reasons"] == []


def test_step_defaults(bench, monkeypatch):
    for argv, steps in ((["bench.py"], 40), (["bench.py", "--workload", "batched"], 40),
                        (["bench.py", "--workload", "gemm"], 3), (["bench.py", "--impl", "reference"], 3),
                        (["bench.py", "--steps", "7"], 7)):
        monkeypatch.setattr(sys, "argv", argv)
        assert bench.parse().steps == steps


def test_oracle_refinement_is_timed_whole(bench):
    from paper_2602_19090_gb300 import synth
    A, X0, D0, _ = synth.refine_workload(96, 1e4, "spd", case=3)
    rec, X, info = bench.cpu_oracle_refine(A, X0, D0, 1e-14)
    assert rec["kind"] == "oracle" and rec["unit"] == "s" and rec["value"] > 0
    assert info["status"] == "converged" and X.shape == (96, 96)
    assert f"{info['iters']} iterations, {info['products']} slice products" in rec["sample"]


def test_reference_arm_reports_the_steps_it_ran(bench, monkeypatch, capsys):
    # each fake oracle refinement "takes" 70 s of a fake clock: with a 180 s budget the arm
    # runs two (the third would end past the budget) and says so, whatever --steps asked
    import json
    clock = [0.0]
    monkeypatch.setattr(bench.time, "perf_counter", lambda: clock[0])

    def fake(A, X0, D0, delta):
        clock[0] += 70.0
        return {"value": 70.0, "unit": "s", "cores": 1, "kind": "oracle", "sample": "fake"}, None, None

    monkeypatch.setattr(bench, "cpu_oracle_refine", fake)
    monkeypatch.setattr(bench, "oracle_warmup", lambda *a: None)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--n", "64", "--steps", "20",
                                      "--warmup", "5", "--ref-budget", "180"])
    bench.run_reference(bench.parse())
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["requested_steps"] == 20
    assert line["ms_per_step"] == 70000.0 and line["value"] == 70.0
    assert line["steps"] * line["ms_per_step"] / 1e3 <= 180


def test_gemm_traffic_only_while_the_kernel_source_matches(bench, tmp_path, monkeypatch):
    # the committed ncu traffic figure is reported only for the kernel it was taken on: a
    # source whose hash differs from the one in the summary gives null
    import hashlib
    import os
    csrc = tmp_path / "paper_2602_19090_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = b"// kernel source as profiled\n"
    (csrc / "gemm_tc.cu").write_bytes(src)
    sha = hashlib.sha256(src).hexdigest()[:16]
    (tmp_path / "profiles" / "plane_gemm_tc256_n4096_traffic.md").write_text(
        f"Average per launch (read + write): traffic_bytes_per_launch: 123456\n"
        f"kernel_source_sha256_16: {sha}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.gemm_traffic() == 123456
    (csrc / "gemm_tc.cu").write_bytes(src + b"// changed\n")
    assert bench.gemm_traffic() is None
    os.remove(csrc / "gemm_tc.cu")
    assert bench.gemm_traffic() is None


def test_job_throughput_is_all_ranks_units_over_the_slowest(bench):
    # 4 ranks, 10 units each, the slowest rank took 2 s: 40 units / 2 s
    assert bench.job_throughput(4, 10, 2000.0) == pytest.approx(20.0)
    assert bench.job_throughput(1, 1, 16.5) == pytest.approx(1e3 / 16.5)
