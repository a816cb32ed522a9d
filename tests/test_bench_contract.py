"""The benchmark's command-line defaults and the reference arm's JSON line (no GPU).

The reference arm is the FP64 oracle on the host cores; its timing is replaced here by a fast
stand-in so that only the line's structure is checked.
"""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _args(monkeypatch, *argv):
    monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
    return bench.parse()


def test_defaults_are_one_gpu_with_three_warmup_steps(monkeypatch):
    a = _args(monkeypatch)
    assert a.gpus == 1 and a.impl == "ours" and a.kernel is None
    assert a.warmup >= 3 and 1 <= a.steps <= 10
    assert a.workload == bench.WORKLOAD


def test_headline_config_names_the_workload():
    c = bench.config_dict()
    assert c["workload"] == bench.WORKLOAD
    assert c["N"] == c["n"] ** c["dim"] and c["tol"] == 1e-8
    assert "flushed" in c["l2"]


def test_reference_line_structure(monkeypatch, capsys):
    calls = []

    def fake_baseline(name, iterations, iterations_from=""):
        calls.append((name, iterations))
        return {"value": 10.0 + len(calls), "unit": "s", "cores": 4, "cpu": "test", "kind": "oracle",
                "sample": "stand-in", "parts_s": {"matvec": 0.1, "apply": 0.01, "factor": 1.0}}

    def fake_full(name, matvec):
        return {"value": 0.5, "unit": "s", "workload": name, "extrapolated": False}
    monkeypatch.setattr(bench, "cpu_baseline", fake_baseline)
    monkeypatch.setattr(bench, "oracle_full_solve", fake_full)
    monkeypatch.delenv("RANK", raising=False)
    a = _args(monkeypatch, "--impl", "reference", "--steps", "2", "--warmup", "3")
    assert bench.run_reference(a) == 0
    assert len(calls) == 5  # three warm-up runs, two timed
    assert all(c[0] == bench.WORKLOAD for c in calls)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "s" and line["higher_is_better"] is False
    assert (line["n_gpus"], line["steps"], line["warmup"]) == (1, 2, 3)
    assert line["value"] == pytest.approx((14.0 + 15.0) / 2)
    assert line["ms_per_step"] == pytest.approx(line["value"] * 1e3)
    assert line["config"]["workload"] == bench.WORKLOAD
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["vs_baseline"] is None and line["data"] == "synthetic"
    # measured (not extrapolated) end-to-end oracle solves ride along: the 64^2 workload every
    # step, the 3D 64-column workload once
    meas = line["cpu_baseline"]["measured_end_to_end"]
    assert set(meas) == {"ie2d_n64_schwarz_m4_d1", "ie3d_n32_schwarz_m4_d1_rhs64"}
    assert all(v["extrapolated"] is False for v in meas.values())


def test_headline_is_the_largest_workload():
    # kernel pairs per matvec: N^2 per right-hand side, over the workloads of the benchmark's
    # configurations (the RS-CBD workloads -- the paper's subdomain solver beyond them -- are legs)
    sizes = {k: (w["n"] ** w["dim"]) ** 2 * w["seeds"] for k, w in bench.WORKLOADS.items() if w["factor"] != "rs"}
    assert bench.WORKLOAD == max(sizes, key=sizes.get) == "ie2d_n1024_schwarz_m64_d2"
    assert {k for k, w in bench.WORKLOADS.items() if w["factor"] == "rs"} == {
        "ie2d_n1024_cbd_rs_m128_d1", "ie2d_n2048_cbd_rs_m256_d1", "ie3d_n64_cbd_rs_m8_d1"}


@pytest.mark.parametrize("clocks,kind", [({"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}, "burst"),
                                         ({"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": []}, "burst"),
                                         ({"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"]},
                                          "sustained"),
                                         ({"sm_mhz": 1440.0, "sm_max_mhz": 2070.0, "reasons": []}, "sustained"),
                                         ({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]},
                                          "sustained")])
def test_tensor_peak_follows_the_clock_record(clocks, kind):
    peak, got = bench.tensor_peak(clocks)
    assert got == kind
    key = "bf16_tflops" if kind == "burst" else "bf16_tflops_sustained"
    assert peak == bench.measured_peak(key, -1.0) or bench.measured_peak(key, -1.0) == -1.0


def test_clock_sampler_parses_samples_and_throttle_reasons(tmp_path, monkeypatch):
    # a stand-in nvidia-smi on PATH prints three samples; the sampler reports the median SM clock,
    # the maximum clock and every throttle reason seen Active
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 1900, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '0, 2070, 2070, 1200.5, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "echo '0, 1500, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    s = bench.ClockSampler(None)
    s.start()
    import time
    for _ in range(100):  # wait until the stand-in has written its samples
        time.sleep(0.05)
        if open(s.path).read().count("\n") >= 3:
            break
    out = s.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 1900.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(None)
    s.start()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]
