"""Host-side logic of bench.py on CPU: the clock / throttle-reason summary of the nvidia-smi
samples (a run with a thermal or hardware slowdown must be visible in the JSON line), the
roofline entry of the dominant kernel from CUDA-event totals and work tallies, and the
per-stage figures."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary(tmp_path, lines):
    s = bench.ClockSampler()
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    return s.summary()


def test_clock_summary_reasons_and_median(tmp_path):
    na, act = "Not Active", "Active"
    lines = [f"0, 2070, 2070, 900.1, 0x0, {na}, {na}, {na}, {na}",
             f"0, 2055, 2070, 1350.0, 0x4, {na}, {na}, {na}, {act}",
             f"0, 1980, 2070, 1400.0, 0x4, {na}, {act}, {na}, {act}",
             "garbage line"]
    out = _summary(tmp_path, lines)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert not os.path.exists(tmp_path / "clocks.csv")


def test_clock_summary_without_samples(tmp_path):
    out = _summary(tmp_path, [])
    assert out["samples"] == 0 and out["reasons"] == ["unavailable"]


def test_roofline_pruned_kernel_from_work_tallies():
    steps = 3
    prof = {"k_nn6d_pruned": (13.0 * steps, 30), "k_fof_link": (6.3 * steps, 6)}
    work = {"nn_d6": 2.8e9, "nn_box": 2.0e9, "link_d6": 1.0e9, "link_box": 1.0e9}
    r = bench._roofline(prof, pairs=4.9e10, steps=steps, work=work)
    peak = bench.SM_COUNT * bench.FP32_LANES_PER_SM * 2070e6
    ops = (2.8e9 + 2.0e9) * bench.OPS_PER_PAIR["k_nn6d"] * steps
    assert r["kernel"] == "k_nn6d_pruned" and r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(ops / (13.0 * steps / 1e3) / 1e12)
    assert r["frac"] == pytest.approx(ops / (13.0 * steps / 1e3) / peak)
    assert r["kernel_ms_per_step"] == pytest.approx(13.0)
    assert r["work"]["d6_per_step"] == 2.8e9


def test_roofline_brute_force_link_counts_unordered_pairs():
    prof = {"k_link6d": (25.0, 10)}
    r = bench._roofline(prof, pairs=4.0e10, steps=1)
    ops = 4.0e10 / 2.0 * bench.OPS_PER_PAIR["k_link6d"]
    assert r["achieved"] == pytest.approx(ops / 25e-3 / 1e12)


def test_stages_entries(monkeypatch):
    monkeypatch.setattr(bench, "_measured_peaks", lambda: {"hbm_gbs": 6761.6})
    r = {"prof": {"k_fof_link": (12.6, 4), "k_link6d_pruned": (15.0, 20)}, "n": 1 << 24,
         "pairs": 4.9e10, "pairs_big": 4.0e10, "form": "surrogate",
         "work": {"nn_d6": 1.0, "nn_box": 1.0, "link_d6": 1.0e9, "link_box": 5.0e8}}
    out = bench._stages(r, steps=2)
    fof = out["k_fof_link"]
    assert fof["bound"] == "hbm"
    assert fof["achieved"] == pytest.approx((1 << 24) * 28.0 / 6.3e-3 / 1e9)
    link = out["k_link6d_pruned"]
    assert link["ms_per_step"] == pytest.approx(7.5)
    assert link["achieved"] == pytest.approx(1.5e9 * 20.0 / 7.5e-3 / 1e12)
    assert "k_potential_blocked" not in out  # the surrogate form's blocked sums are partial
