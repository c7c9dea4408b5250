"""Host logic of bench.py's measurement record (no GPU): the committed ncu traffic record, its lookup
by kernel source hash and launch shape, and the peak used as the roofline denominator."""
import json
import os
import shutil

import pytest

import bench

KEYS = {"kernel", "kernel_sha", "variant", "bvh", "tuning", "workload", "rays", "dram_read_bytes",
        "dram_write_bytes", "dram_bytes", "command"}
TUNING_KEYS = {"tile_w", "tile_h", "persistent", "terrain_first", "min_blocks"}


def test_traffic_record_is_well_formed():
    with open(bench.TRAFFIC) as f:
        caps = json.load(f)["captures"]
    assert caps
    for c in caps:
        assert KEYS <= set(c), c
        assert set(c["tuning"]) == TUNING_KEYS
        assert c["tuning"]["tile_w"] * c["tuning"]["tile_h"] == 32
        assert c["dram_bytes"] == c["dram_read_bytes"] + c["dram_write_bytes"]
        assert c["rays"] > 0 and c["dram_bytes"] > 0
        assert c["variant"] in ("plain", "precision", "perception", "batching")
        # the command re-creates the capture from committed files only, with unlocked clocks
        assert c["command"].startswith("ncu --set full --clock-control none ")
        assert " python bench.py " in c["command"] and "_work" not in c["command"]
        t = c["tuning"]
        assert c["command"].endswith("--tuning %d,%d,%d,%d,%d" % (t["tile_w"], t["tile_h"], t["persistent"],
                                                                   t["terrain_first"], t["min_blocks"]))


def test_traffic_lookup_matches_hash_shape_and_layout(tmp_path, monkeypatch):
    tuning = {"tile_w": 4, "tile_h": 8, "persistent": 0, "terrain_first": 0, "min_blocks": 12}
    rec = {"captures": [{"kernel_sha": bench.kernel_hash(), "variant": "plain", "bvh": 2, "tuning": tuning,
                         "rays": 1000, "dram_bytes": 5000},
                        {"kernel_sha": "0" * 16, "variant": "perception", "bvh": 2, "tuning": tuning,
                         "rays": 10, "dram_bytes": 10}]}
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC", str(p))
    # scaled to a launch of 4000 rays
    assert bench.traffic_per_launch(4000, "plain", tuning, 2) == pytest.approx(20000.0)
    # another shape, layout or variant, or a capture of other kernel sources: no figure
    assert bench.traffic_per_launch(4000, "plain", dict(tuning, min_blocks=10), 2) is None
    assert bench.traffic_per_launch(4000, "plain", tuning, 8) is None
    assert bench.traffic_per_launch(4000, "precision", tuning, 2) is None
    assert bench.traffic_per_launch(4000, "perception", tuning, 2) is None
    monkeypatch.setattr(bench, "TRAFFIC", str(tmp_path / "missing.json"))
    assert bench.traffic_per_launch(4000, "plain", tuning, 2) is None


def test_kernel_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2602_03002_gb300", "csrc")
    dst = tmp_path / "paper_2602_03002_gb300" / "csrc"
    shutil.copytree(src, dst, ignore=shutil.ignore_patterns("*.o", "*.so"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_hash()
    assert h0 == bench.kernel_hash()
    f = dst / "render.cu"
    text = f.read_text()
    f.write_text("// a new comment line\n\n" + text.replace("{", "{  // trailing comment", 1))
    assert bench.kernel_hash() == h0
    f.write_text(text + "\nstatic int an_extra_symbol;\n")
    assert bench.kernel_hash() != h0


def test_peak_comes_from_the_measured_file(tmp_path, monkeypatch):
    p = tmp_path / "peaks.json"
    p.write_text(json.dumps({"hbm_gbs": 6777.3}))
    monkeypatch.setattr(bench, "PEAKS", str(p))
    assert bench.peaks() == (6777.3, "measured")
    monkeypatch.setattr(bench, "PEAKS", str(tmp_path / "absent.json"))
    assert bench.peaks() == (6800.0, "fallback")
