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


def _form(**kw):
    r = {"n": 1 << 24, "members": 15_000_000, "sort_keypasses": 4 * (1 << 24),
         "pairs": {"pairs_all": 4.9e10, "pairs_small": 1.0e9, "pairs_blocked": 3.0e10},
         "work": {"nn_d6": 2.8e9, "nn_box": 2.0e9, "link_d6": 1.0e9, "link_box": 1.0e9},
         "tree": {"expansions": 2.0e9, "direct_pairs": 5.0e9, "list_pairs": 1.0e10}}
    r.update(kw)
    return r


def test_stages_use_the_per_unit_figures(monkeypatch):
    monkeypatch.setattr(bench, "_measured_peaks", lambda: {"hbm_gbs": 6700.0})
    prof = {"k_fof_link": (6.0, 2), "k_sort_hist": (1.0, 40), "k_sort_scatter": (3.0, 40),
            "k_nn6d_pruned": (13.0, 20), "k_potential_list": (5.0, 3), "k_tree_walk": (8.0, 3),
            "k_potential_blocked": (2.0, 1)}
    st = bench.stages(_form(prof=prof))
    fof = st["k_fof_link"]
    assert fof["bound"] == "hbm" and fof["unit"] == "GB/s"
    assert fof["achieved"] == pytest.approx((1 << 24) * 28.0 / 6.0e-3 / 1e9)
    assert fof["frac"] == pytest.approx(fof["achieved"] / 6700.0)
    srt = st["k_sort"]
    assert srt["ms_per_step"] == 4.0 and srt["launches"] == 80
    assert srt["achieved"] == pytest.approx(4 * (1 << 24) * 24.0 / 4.0e-3 / 1e9)
    nn = st["k_nn6d_pruned"]
    assert nn["bound"] == "hbm"
    assert nn["achieved"] == pytest.approx(15e6 * 40.0 / 13e-3 / 1e9)
    assert nn["alu_d6_only"]["achieved"] == pytest.approx(2.8e9 * 20.0 / 13e-3 / 1e12)
    lst = st["k_potential_list"]
    assert lst["bound"] == "alu"
    assert lst["achieved"] == pytest.approx(1.0e10 * 7.0 / 5e-3 / 1e12)
    assert st["k_tree_walk"]["achieved"] == pytest.approx((2e9 * 50 + 5e9 * 7) / 8e-3 / 1e12)
    assert st["k_potential_blocked"]["achieved"] == pytest.approx(3e10 * 7 / 2e-3 / 1e12)


def test_roofline_is_the_dominant_kernel_with_traffic(monkeypatch):
    monkeypatch.setattr(bench, "_measured_peaks", lambda: {"hbm_gbs": 6700.0})
    prof = {"k_fof_link": (6.0, 2), "k_nn6d_pruned": (13.0, 20), "k_unknown": (99.0, 1)}
    r = bench.roofline(_form(prof=prof), traffic={"k_nn6d_pruned": 1.5e9})
    assert r["kernel"] == "k_nn6d_pruned" and r["traffic"] == 1.5e9
    assert r["ms_per_launch"] == pytest.approx(13.0 / 20)
    assert r["peak"] == 6700.0 and r["peak_source"] == "measured"


def test_brute_force_pairs_and_form_thresholds():
    sizes = [10, 300, 500, 2000, 20000]
    p = bench._sizes_work(sizes, "plain", 0)
    pair = lambda g: g * (g - 1.0)  # noqa: E731
    assert p["pairs_small"] == pair(10) + pair(300)
    assert p["pairs_blocked"] == pair(500) + pair(2000) + pair(20000)
    b = bench._sizes_work(sizes, "batched", 16384)
    assert b["pairs_blocked"] == pair(500) + pair(2000)
    s = bench._sizes_work(sizes, "surrogate", 16384)
    assert s["pairs_blocked"] == pair(500)
    r = _form(pairs=p, prof={"k_link6d": (25.0, 10)})
    assert bench._alu_d6(r, "k_link6d") == pytest.approx(p["pairs_all"] / 2 * 20.0)


def test_oracle_sample_cubes_around_the_median_load():
    L = 80.0
    cat = []
    # one top-level halo per cube on the diagonal of 8 cubes, loads 1..8 squared; one subhalo
    for i in range(8):
        c = (i + 0.5) * L / 8
        cat.append((0, i + 1, i + 1, (c, c, c), (0, 0, 0), 1.0))
    cat.append((1, 1000, 1000, (5.0, 5.0, 5.0), (0, 0, 0), 1.0))   # depth 1: ignored
    snap = {"box": L, "catalogue": cat}
    cubes = bench._oracle_cubes(snap, count=3)
    assert len(cubes) == 3
    # 504 empty cubes sort first, so the median of the 512 lies among the empty ones
    assert all(c not in [(i, i, i) for i in range(8)] for c in cubes)
    loads = {(i, i, i): (i + 1) ** 2 for i in range(8)}
    assert all(loads.get(c, 0) == 0 for c in cubes)


def test_six_d_stages_follow_the_form(monkeypatch):
    """The batched forms run the brute-force pair kernels only on their small levels: those get
    no stage entry there (the per-member figure would not describe them); the plain form reports
    them and no pruned kernel."""
    monkeypatch.setattr(bench, "_measured_peaks", lambda: {"hbm_gbs": 6700.0})
    prof = {"k_nn6d": (4.0, 5), "k_link6d": (2.0, 5), "k_nn6d_pruned": (13.0, 20),
            "k_link6d_pruned": (7.0, 10)}
    batched = bench.stages(_form(prof=prof, form="batched"))
    assert "k_nn6d_pruned" in batched and "k_link6d_pruned" in batched
    assert "k_nn6d" not in batched and "k_link6d" not in batched
    plain = bench.stages(_form(prof=prof, form="plain"))
    assert "k_nn6d" in plain and "k_link6d" in plain and "k_nn6d_pruned" not in plain


def test_traffic_attached_to_stages(monkeypatch):
    monkeypatch.setattr(bench, "_measured_peaks", lambda: {"hbm_gbs": 6700.0})
    prof = {"k_fof_link": (6.0, 2), "k_tree_walk": (8.0, 3)}
    st = bench.stages(_form(prof=prof), {"k_fof_link": 3.0e9, "k_tree_walk": 7.0e8})
    assert st["k_fof_link"]["traffic"] == 3.0e9
    assert st["k_fof_link"]["algorithmic_bytes_per_launch"] == pytest.approx((1 << 24) * 28.0 / 2)
    assert st["k_tree_walk"]["traffic"] == 7.0e8 and "algorithmic_bytes_per_launch" not in st["k_tree_walk"]


def test_stream_snapshots_follow_the_recipe():
    """The batched stream's snapshot k has n = 2^(18 + k mod 5) particles at unit mean spacing
    (box = n^(1/3)); the generator worker returns what the pipeline needs."""
    from paper_2412_18629_gb300 import synth
    for k in range(7):
        spec = synth.stream_spec(k)
        assert spec.n == 1 << (18 + k % 5)
        assert spec.box == pytest.approx(spec.n ** (1.0 / 3.0), rel=1e-12)
    s = bench._gen_stream(0)
    assert set(s) == {"pos", "vel", "ids", "box", "link_length", "softening", "particle_mass"}
    assert s["pos"].shape == (1 << 18, 3) and s["ids"].dtype.name == "int64"
