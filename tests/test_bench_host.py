"""Host logic of the benchmark, without a GPU: the clock record that decides
whether a run is kept (median SM clock, throttle reasons) and the FP64 peak
derivation."""
import os

import pytest

pytest.importorskip("torch")

import bench  # noqa: E402


def _clocks_from(tmp_path, lines):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    c.proc = object()   # as if nvidia-smi had been started
    return c.summary()


def test_clock_summary_median_and_reasons(tmp_path):
    rows = [
        "0, 2070, 2070, 690.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 705.3, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 701.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 700.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = _clocks_from(tmp_path, rows)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_hw_slowdown(tmp_path):
    rows = ["0, 1500, 2070, 900.0, 0x48, Active, Not Active, Active, Not Active"]
    s = _clocks_from(tmp_path, rows)
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1500.0


def test_clock_summary_without_samples(tmp_path):
    assert _clocks_from(tmp_path, [])["reasons"] == ["no samples"]
    c = bench.Clocks(0)
    c.proc = None
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_fp64_peak_derivation(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))      # no MEASURED_PEAKS.json there
    peak, how = bench.fp64_peak(152)
    assert peak == pytest.approx(152 * 4 * 2070e6 / 1e12) and "152 SMs" in how
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"sm_max_mhz": 1980.0}')
    assert bench.fp64_peak(152)[0] == pytest.approx(152 * 4 * 1980e6 / 1e12)
    assert os.path.exists(tmp_path / "MEASURED_PEAKS.json")


def test_cpu_oracle_legs_small():
    """The host-core legs of the benchmark on a tiny case: config 1's full
    oracle solve converges to 1e-10, and the one-core and all-core operator
    rates are positive with the core count stated."""
    out = bench.cpu_legs(orders=(3,), k=2, reps=1)
    c1 = out["config1_fp64_pcg_to_1e-10"]
    assert c1["relres"] <= 1e-10 and 0 < c1["iterations"] < 500
    (leg,) = out["config3_ax"]
    assert leg["N"] == 3 and leg["local_dofs_per_process"] == 8 * 64
    assert leg["gdofs_1core"] > 0 and leg["gdofs_all_cores"] > 0
    assert leg["cores"] == out["cores_available"] >= 1
