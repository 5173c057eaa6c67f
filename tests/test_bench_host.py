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


def test_class_butterflies():
    n = 1 << bench.LOGN
    half = (bench.LOGN // 2) * (n / 2)
    assert bench.class_butterflies("ntt_fwd", 3, 0) == pytest.approx(3 * 2 * half)
    assert bench.class_butterflies("modup", 5, 2) == pytest.approx(7 * half)
    assert bench.class_butterflies("ks_inner", 4, 99) == pytest.approx(4 * half)


def _traffic_file(tmp_path, body):
    (tmp_path / "profiles").mkdir(exist_ok=True)
    (tmp_path / "profiles" / "traffic.txt").write_text(body)


def test_keyswitch_traffic_and_pipe_records(tmp_path, monkeypatch):
    _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_sources_hash()
    _traffic_file(tmp_path, "# comment keyswitch %s nl=7 1.0\n"
                            "keyswitch %s nl=7 700.0\n"
                            "keyswitch %s nl=4 400.0\n"
                            "keyswitch 000000000000 nl=5 9.0\n"
                            "fmaheavy k_ks_modup_cols %s 15.9\n"
                            "fmaheavy k_ks_inner_rows 000000000000 3.0\n" % (h, h, h, h))
    # weighted by the key switches of each limb count
    assert bench.recorded_keyswitch_traffic({7: 1, 4: 3}) == pytest.approx((700 + 3 * 400) / 4)
    assert bench.recorded_keyswitch_traffic({7: 1, 5: 1}) is None  # no record for 5 limbs at this hash
    assert bench.recorded_keyswitch_traffic({}) is None
    assert bench.recorded_fmaheavy("k_ks_modup_cols") == pytest.approx(15.9)
    assert bench.recorded_fmaheavy("k_ks_inner_rows") is None
    # a whole-iteration record serves any mix of limb counts
    _traffic_file(tmp_path, "keyswitch %s nl=all 36.0e6\nkeyswitch %s nl=7 1.0\n" % (h, h))
    assert bench.recorded_keyswitch_traffic({7: 1, 5: 2}) == pytest.approx(36.0e6)


def test_roofline_of_the_key_switch(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 7000.0})
    monkeypatch.setattr(bench, "recorded_keyswitch_traffic", lambda by: 2.0e6)
    rec = {"k_ks_modup_cols": 16.0}
    monkeypatch.setattr(bench, "recorded_fmaheavy", lambda k: rec.get(k))
    n = 1 << bench.LOGN
    # (ms, units, launches, units2, dram_limbs) per class over 2 steps
    prof = {"ntt_fwd": (100.0, 10, 4, 0, 0), "ntt_inv": (50.0, 5, 2, 0, 0),
            "modup": (400.0, 100, 8, 20, 300), "ks_inner": (300.0, 90, 8, 500, 200)}
    ks = (800.0, 40, 0, 200, 1000)  # 40 key switches, 1000 algorithmic limbs, 0.8 s
    r = bench.roofline(prof, ks, {5: 40}, 2, 0.5, 152, 2070.0)
    alg = 1000 * 8.0 * n
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 7000.0
    assert r["achieved"] == pytest.approx(round(alg / 0.8 / 1e9, 1))
    assert r["frac"] == pytest.approx(alg / 0.8 / 1e9 / 7000.0, abs=1e-4)
    assert r["alg_bytes_per_unit"] == round(alg / 40) and r["traffic"] == 2000000
    assert r["keyswitch_hbm_frac_of_iteration"] == pytest.approx(alg / 2 / 0.5 / 1e9 / 7000.0, abs=1e-4)
    assert r["share_of_step"] == pytest.approx(0.8)
    assert r["keyswitches_by_limbs"] == {"5": 20}
    assert r["dominant_class"] == "modup" and r["dominant_share"] == pytest.approx(round(400 / 850, 3))
    iv = r["issue_view"]
    bf = bench.class_butterflies("modup", 100, 20)
    peak = 152 * 64 * 2070e6 / 32
    assert iv["kernel"] == "k_ks_modup_cols"
    assert iv["frac"] == pytest.approx(bf / 32 * 16.0 / 0.4 / peak, abs=1e-4) and iv["sms"] == 152
    assert r["classes_ms_per_step"] == {"ntt_fwd": 50.0, "ntt_inv": 25.0, "modup": 200.0, "ks_inner": 150.0}
    # without an instruction record for the column kernel there is no issue view
    rec.clear()
    assert bench.roofline(prof, ks, {5: 40}, 2, 0.5, 152, 2070.0)["issue_view"] is None


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
