"""Host logic of bench.py that needs no GPU: the recorded-traffic lookup of
the roofline (plan match and source-region digest)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_recorded_traffic_matches_only_its_plan_distribution_and_source(tmp_path,
                                                                        monkeypatch):
    """The committed record's shape, then the lookup on a copy of it whose
    digest is made to match a source file of the test's own: the traffic is
    returned only for the recorded distribution and plan, and only while the
    source region is unchanged."""
    rec = json.load(open(os.path.join(ROOT, "profiles", "k_tile_normal_skew_large_traffic.json")))
    assert rec["traffic_bytes"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_text("// BEGIN\nkernel body\n// END\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec["sources"] = [{"file": "k.cu", "from": "// BEGIN", "to": "// END"}]
    rec["source_sha256"] = bench.source_digest(rec["sources"])
    (tmp_path / "profiles" / "k_tile_normal_skew_large_traffic.json").write_text(json.dumps(rec))
    plan = dict(rec["plan"], q_tiles=0, split=0, n_block=0, tc_min_row_nnz=0)
    assert bench.recorded_traffic(rec["dist"], plan) == rec["traffic_bytes"]
    other = dict(plan, panel_rows=plan["panel_rows"] // 2)
    assert bench.recorded_traffic(rec["dist"], other) is None
    assert bench.recorded_traffic("uniform" if rec["dist"] != "uniform" else "normal",
                                  plan) is None
    (tmp_path / "k.cu").write_text("// BEGIN\nkernel body changed\n// END\n")
    assert bench.recorded_traffic(rec["dist"], plan) is None


def test_source_digest_covers_exactly_its_region(tmp_path, monkeypatch):
    f = tmp_path / "k.cu"
    f.write_text("head\n// BEGIN here\nbody 1\nbody 2\n// END\ntail\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    region = [{"file": "k.cu", "from": "// BEGIN", "to": "// END"}]
    d0 = bench.source_digest(region)
    f.write_text("head changed\n// BEGIN here\nbody 1\nbody 2\n// END\ntail changed\n")
    assert bench.source_digest(region) == d0          # outside the region
    f.write_text("head\n// BEGIN here\nbody 1\nbody 3\n// END\ntail\n")
    assert bench.source_digest(region) != d0          # inside the region
    whole = [{"file": "k.cu"}]
    assert bench.source_digest(whole) != bench.source_digest(region)
