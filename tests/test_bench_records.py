"""The DRAM-traffic records behind the bench line's `roofline.traffic`: every
record names a committed ncu summary whose table holds the bytes it states and
whose header names the kernel build (source hash) it was taken of, and the bench
reports a record only for the kernel sources it was captured from."""
import json
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")


def _entries():
    return json.load(open(TRAFFIC))["entries"]


def _launch_rows(md):
    """(read + write) MB of every launch row of a summary's traffic table."""
    rows = []
    for line in md.splitlines():
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) >= 4 and cells[0].isdigit() and all(c.endswith("MB") for c in cells[1:4]):
            rows.append(float(cells[3].split()[0]))
    return rows


@pytest.mark.parametrize("i", range(len(_entries())))
def test_traffic_record_traces_to_its_profile(i):
    e = _entries()[i]
    path = os.path.join(ROOT, e["profile"])
    assert os.path.isfile(path), e["profile"]
    md = open(path).read()
    assert e["source_hash"] in md
    assert e["kernel"] in md
    assert re.fullmatch(r"[0-9a-f]{16}", e["source_hash"])
    rows = _launch_rows(md)
    assert len(rows) == e["launches_captured"]
    mean_mb = sum(rows) / len(rows)
    assert abs(mean_mb - e["dram_bytes_per_launch"] / 1e6) <= 0.05 + 1e-4 * mean_mb, (mean_mb, e)


def test_traffic_records_are_unique():
    keys = [(e["workload"], e.get("side"), e["precision"], e["kernel"]) for e in _entries()]
    assert len(keys) == len(set(keys))


def test_bench_reports_traffic_only_for_the_captured_sources(tmp_path, monkeypatch):
    import bench
    from paper_2209_08001_gb300 import build
    h = build.source_hash("k_ras_apply_lane")
    rec = {"entries": [
        {"workload": "w1", "side": None, "precision": "mixed", "kernel": "k_ras_apply_lane", "source_hash": h,
         "dram_bytes_per_launch": 123, "launches_captured": 1, "profile": "profiles/x.md"},
        {"workload": "w2", "side": None, "precision": "mixed", "kernel": "k_ras_apply_lane",
         "source_hash": "0" * 16 if h != "0" * 16 else "1" * 16, "dram_bytes_per_launch": 456,
         "launches_captured": 1, "profile": "profiles/y.md"}]}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    tr, why = bench.traffic_for("w1", None, "mixed", "k_ras_apply_lane")
    assert tr == 123 and "profiles/x.md" in why
    tr, why = bench.traffic_for("w2", None, "mixed", "k_ras_apply_lane")
    assert tr is None and h in why and "profiles/y.md" in why
    tr, why = bench.traffic_for("w1", None, "fp64", "k_ras_apply_lane")
    assert tr is None and "no ncu traffic record" in why
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.json"))
    tr, why = bench.traffic_for("w1", None, "mixed", "k_ras_apply_lane")
    assert tr is None


def test_roofline_of_the_sweep_is_algorithmic_bytes_over_the_mean_launch_time():
    import bench
    st = {"ms": {"schwarz_apply": 20.0, "jacobian_action": 5.0}, "launches": {"schwarz_apply": 40,
                                                                             "jacobian_action": 40},
          "schwarz_bytes": 2.0e9, "schwarz_flops": 1.0e9}
    pk = {"hbm_gbs": 5000.0, "source": "test peaks"}
    r = bench.roofline(st, {}, True, pk, "no-such-workload", None, "mixed")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["avg_launch_ms"] == pytest.approx(0.5)
    assert r["achieved"] == pytest.approx(2.0e9 / 0.5e-3 / 1e9)  # 4000 GB/s
    assert r["frac"] == pytest.approx(0.8)
    assert r["traffic"] is None and r["launches"] == 40
    r64 = bench.roofline(st, {}, False, pk, "no-such-workload", None, "fp64")
    assert r64["unit"] == "TFLOP/s"
    assert r64["achieved"] == pytest.approx(1.0e9 / 0.5e-3 / 1e12)
    assert r64["frac"] == pytest.approx(r64["achieved"] / bench.FP64_PEAK_TFLOPS)
