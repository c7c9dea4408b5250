"""Host logic of bench.py's measurement record (no GPU): the committed ncu counter record, its lookup by
kernel source hash, launch shape and workload size, the roofline against the binding resource, and
the peak used as the HBM denominator."""
import json
import os
import shutil

import pytest

import bench

KEYS = {"kernel", "kernel_sha", "variant", "bvh", "tuning", "workload", "rays", "dram_read_bytes",
        "dram_write_bytes", "dram_bytes", "lts_bytes", "inst_executed", "command"}
TUNING_KEYS = {"tile_w", "tile_h", "persistent", "terrain_first", "min_blocks", "env_order", "chunk_envs"}


def test_counter_record_is_well_formed():
    with open(bench.COUNTERS) as f:
        caps = json.load(f)["captures"]
    assert caps
    for c in caps:
        assert KEYS <= set(c), c
        assert set(c["tuning"]) == TUNING_KEYS
        assert c["tuning"]["tile_w"] * c["tuning"]["tile_h"] == 32
        assert c["dram_bytes"] == c["dram_read_bytes"] + c["dram_write_bytes"]
        assert c["rays"] > 0 and c["dram_bytes"] > 0 and c["lts_bytes"] > 0 and c["inst_executed"] > 0
        assert c["variant"] in ("plain", "precision", "perception", "batching")
        # the command re-creates the capture from committed files only, with unlocked clocks, on one
        # launch of the bench's own full-size workload in the same launch shape
        assert c["command"].startswith("ncu --metrics ") and " --clock-control none " in c["command"]
        assert " -c 1 " in c["command"] and " python bench.py " in c["command"] and "_work" not in c["command"]
        assert "--envs" not in c["command"]
        t = c["tuning"]
        assert c["command"].endswith("--tuning %d,%d,%d,%d,%d,%d,%d" % (
            t["tile_w"], t["tile_h"], t["persistent"], t["terrain_first"], t["min_blocks"], t["env_order"],
            t["chunk_envs"]))


def test_counter_lookup_matches_hash_shape_layout_and_size(tmp_path, monkeypatch):
    tuning = {"tile_w": 4, "tile_h": 8, "persistent": 2, "terrain_first": 0, "min_blocks": 8, "env_order": 1,
              "chunk_envs": 0}
    rec = {"captures": [{"kernel_sha": bench.kernel_hash(), "variant": "plain", "bvh": 2, "tuning": tuning,
                         "rays": 1000, "dram_bytes": 5000, "lts_bytes": 9000, "inst_executed": 77},
                        {"kernel_sha": "0" * 16, "variant": "perception", "bvh": 2, "tuning": tuning,
                         "rays": 10, "dram_bytes": 10, "lts_bytes": 10, "inst_executed": 1}]}
    p = tmp_path / "counters.json"
    p.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "COUNTERS", str(p))
    assert bench.counters_for_launch(1000, "plain", tuning, 2)["dram_bytes"] == 5000
    # another size (no scaling), shape, layout or variant, or other kernel sources: no figure
    assert bench.counters_for_launch(4000, "plain", tuning, 2) is None
    assert bench.counters_for_launch(1000, "plain", dict(tuning, min_blocks=10), 2) is None
    assert bench.counters_for_launch(1000, "plain", tuning, 8) is None
    assert bench.counters_for_launch(1000, "precision", tuning, 2) is None
    assert bench.counters_for_launch(10, "perception", tuning, 2) is None
    monkeypatch.setattr(bench, "COUNTERS", str(tmp_path / "missing.json"))
    assert bench.counters_for_launch(1000, "plain", tuning, 2) is None


def test_roofline_names_the_highest_fraction(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: (6800.0, "measured"))
    cnt = {k: 1.0 for k in ("terrain_nodes", "terrain_tris", "link_boxes", "link_nodes", "link_tris")}
    ctr = {"dram_bytes": 3.4e9, "lts_bytes": 20e9, "inst_executed": 2.0e9}
    # 1 ms: DRAM 3400 GB/s (0.5), L2 20000 of 40000 GB/s (0.5), issue 2000 of 152*4*2.07 = 1258.56 G/s
    r = bench.roofline(ctr, 1e-3, 900.0 * 1e6, 1e6, 152, 2070.0, 40000.0, cnt)
    assert r["hbm"]["frac"] == pytest.approx(0.5) and r["l2"]["frac"] == pytest.approx(0.5)
    assert r["issue"]["frac"] == pytest.approx(2000.0 / 1258.56)
    assert r["bound"] == "issue" and r["frac"] == r["issue"]["frac"] and r["traffic"] == 3.4e9
    assert r["fetch_bytes_per_ray"] == pytest.approx(900.0)
    r = bench.roofline(dict(ctr, inst_executed=1e8), 1e-3, 9e8, 1e6, 152, 2070.0, 80000.0, cnt)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["frac"] == pytest.approx(0.5)
    r = bench.roofline(None, 1e-3, 9e8, 1e6, 152, 2070.0, 80000.0, cnt)
    assert r["frac"] is None and r["traffic"] is None and r["bound"] is None


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
