"""Host-side logic of bench.py on CPU: the roofline arithmetic of the bench
line, the source hash that keys the recorded DRAM traffic, the traffic record
lookup and the parsing of the clock samples."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

SRC = ("ntt_core.cuh", "ks.cu", "ntt.cu")


def _copy_sources(tmp_path):
    d = tmp_path / "paper_2406_13221_gb300" / "csrc"
    d.mkdir(parents=True)
    for f in SRC:
        shutil.copy(os.path.join(ROOT, "paper_2406_13221_gb300", "csrc", f), d / f)
    return d


def test_kernel_hash_ignores_comments_and_whitespace(tmp_path, monkeypatch):
    d = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_sources_hash()
    ks = d / "ks.cu"
    text = ks.read_text()
    ks.write_text("// a new leading comment\n/* and a\n   block comment */\n" + text.replace("\n", "\n\n", 3))
    assert bench.kernel_sources_hash() == h0
    # a change of code changes the hash
    ks.write_text(text.replace("CH = 4", "CH = 2", 1))
    assert "CH = 4" in text
    assert bench.kernel_sources_hash() != h0


def test_recorded_traffic_lookup(tmp_path, monkeypatch):
    _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_sources_hash()
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.txt").write_text(
        "# kernel hash ratio\n"
        "# k_ks_modup_cols %s 9.9 commented out\n"
        "k_ks_modup_cols 000000000000 5.0 other sources\n"
        "k_ks_modup_cols %s 0.9227 items=32\n"
        "k_ks_inner_rows 000000000000 1.01 other sources\n" % (h, h))
    assert bench.recorded_traffic("k_ks_modup_cols") == pytest.approx(0.9227)
    assert bench.recorded_traffic("k_ks_inner_rows") is None  # recorded for other sources only
    assert bench.recorded_traffic("k_unknown") is None


def test_class_work_counts():
    n = 1 << bench.LOGN
    half = (bench.LOGN // 2) * (n / 2) * bench.OPS_BFLY
    ops, byt = bench.class_work("ntt_fwd", 3, 0, 0)
    assert ops == pytest.approx(3 * 2 * half) and byt == pytest.approx(3 * 16.0 * n)
    ops, byt = bench.class_work("modup", 5, 2, 11)
    assert ops == pytest.approx(5 * (half + n * bench.OPS_LIFT) + 2 * (half + n * bench.OPS_SCALE))
    assert byt == pytest.approx(11 * 8.0 * n)
    ops, byt = bench.class_work("ks_inner", 4, 7, 9)
    assert ops == pytest.approx(4 * half + 7 * n * bench.OPS_MAC) and byt == pytest.approx(9 * 8.0 * n)


def test_roofline_picks_the_slowest_class(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 7000.0})
    monkeypatch.setattr(bench, "recorded_traffic", lambda k: 0.5 if k == "k_ks_modup_cols" else None)
    # (ms, units, launches, units2, dram_limbs) per class over 2 steps
    prof = {"ntt_fwd": (100.0, 10, 4, 0, 0), "ntt_inv": (50.0, 5, 2, 0, 0),
            "modup": (400.0, 100, 8, 20, 300), "ks_inner": (300.0, 90, 8, 500, 200)}
    r = bench.roofline(prof, 2)
    assert r["kernel"] == "k_ks_modup_cols" and r["bound"] == "alu" and r["launches"] == 8
    ops, byt = bench.class_work("modup", 100, 20, 300)
    peak = bench.SMS * bench.LANES * bench.SM_MHZ_MAX * 1e6 / 1e12
    assert r["peak"] == pytest.approx(round(peak, 2))
    assert r["achieved"] == pytest.approx(round(ops / 0.4 / 1e12, 2))
    assert r["frac"] == pytest.approx(ops / 0.4 / 1e12 / peak, abs=1e-4)
    assert r["traffic"] == round(0.5 * byt / 8)  # the record's ratio scaled to one average launch
    assert r["hbm_view"]["achieved"] == pytest.approx(round(byt / 0.4 / 1e9, 1))
    assert r["share_of_timed_classes"] == pytest.approx(round(400 / 850, 3))
    assert r["classes_ms_per_step"] == {"ntt_fwd": 50.0, "ntt_inv": 25.0, "modup": 200.0, "ks_inner": 150.0}
    # without a record for the dominant kernel the traffic is null
    prof["ks_inner"] = (500.0, 90, 8, 500, 200)
    assert bench.roofline(prof, 2)["traffic"] is None


def test_transform_limbs_counts_halves():
    # (ms, units, launches, units2, dram_limbs): fused kernels report halves (ModUp:
    # forward column halves in units, inverse column halves in units2)
    prof = {"ntt_fwd": (0, 3, 0, 0, 0), "ntt_inv": (0, 2, 0, 0, 0),
            "modup": (0, 10, 0, 6, 0), "ks_inner": (0, 8, 0, 0, 0)}
    assert bench.transform_limbs(prof) == pytest.approx(3 + 2 + 0.5 * (10 + 6 + 8))


def test_clock_samples_are_parsed(tmp_path):
    csv = tmp_path / "clocks.csv"
    csv.write_text(
        "index, clocks.current.sm [MHz], clocks.max.sm [MHz], power.draw [W], active, hw, hwt, swt, swpc\n"
        "0, 2070, 2070, 700.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
        "0, 2055, 2070, 810.0, 0x4, Not Active, Not Active, Not Active, Active\n"
        "0, 2070, 2070, 790.2, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    c = bench.clocks_stop((None, str(csv)))
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"] and c["power_w_max"] == pytest.approx(810.0)
    assert not csv.exists()
    assert bench.clocks_stop((None, str(tmp_path / "missing.csv")))["reasons"] == ["unavailable"]
