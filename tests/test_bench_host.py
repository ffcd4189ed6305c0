"""Host-side logic of bench.py on the CPU: the algorithmic flop convention and the parsing of the
clock samples that decide whether a timed run is kept (throttle reasons, median SM clock)."""
import tempfile

import pytest

import bench


def test_algorithmic_flops_convention():
    # two windows: (m, M) = (3, 5) and (2, 4); N = 5, K = 2
    plan = [[0, 3], [3, 2], [0, 1], [5, 4]]
    f = bench.algorithmic_flops(plan, 5, 2)
    eig = 4.0 / 3.0 * 5 ** 3 + 2.0 * 25 * 3 + 4.0 / 3.0 * 4 ** 3 + 2.0 * 16 * 2
    fs = 2.0 * 5 * (5 * 3 + 4 * 2) + 2.0 * 125 + 1 * 4.0 * 125
    gs = 125 + 125 / 3.0 + 125
    assert f["eig"] == pytest.approx(eig)
    assert f["fs"] == pytest.approx(fs)
    assert f["gs"] == pytest.approx(gs)
    assert f["rayleigh"] == pytest.approx(250.0)
    assert f["total"] == pytest.approx(eig + fs + gs + 250.0)
    assert bench.algorithmic_flops(plan, 5, 0)["fs"] == 0.0


def test_window_reduction_flops_of_the_bench_workload():
    # ten windows of 384 rows: the k_tridiag roofline's 4/3 M^3 per window
    plan = [[0] * 10, [128] * 10, [0] * 10, [384] * 10]
    f = bench.algorithmic_flops(plan, 1280, 3)
    assert f["eig"] - 10 * 2.0 * 384 * 384 * 128 == pytest.approx(754974720.0)


def _smi_sampler(lines):
    s = bench.ClockSampler(0)
    s.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    s.f.write("\n".join(lines) + "\n")
    return s


def test_clock_samples_from_nvidia_smi():
    row = "0, {sm}, 2032, 950.0, 0x{act:016x}, {hw}, Not Active, Not Active, {cap}"
    s = _smi_sampler([row.format(sm=2032, act=0, hw="Not Active", cap="Not Active"),
                      row.format(sm=2020, act=4, hw="Not Active", cap="Active"),
                      row.format(sm=2032, act=0, hw="Not Active", cap="Not Active")])
    out = s.summary()
    assert out["sm_mhz"] == 2032.0 and out["sm_max_mhz"] == 2032.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]                 # kept and noted
    s = _smi_sampler([row.format(sm=1500, act=8, hw="Active", cap="Not Active")])
    assert s.summary()["reasons"] == ["hw_slowdown"]          # a run that is rejected


def test_clock_samples_from_nvml():
    s = bench.ClockSampler(0)
    s.nvml = (None, None)
    s.rows = [(2032.0, 2032.0, 0x0), (2032.0, 2032.0, 0x4 | 0x40), (1900.0, 2032.0, 0x0)]
    out = s.summary()
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert out["sm_mhz"] == 2032.0 and out["samples"] == 3
    s.rows = []
    assert s.summary()["reasons"] == ["unsampled"]


def test_job_rate_counts_every_rank():
    assert bench.job_rate(20, 4, 2.0) == 40.0
