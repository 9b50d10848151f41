"""Host-side logic of bench.py without a GPU: the algorithmic operation count
per ray, the optics variants of a workload (per-frame copies, nothing
applied twice), the roofline arithmetic and the guard that drops a DRAM
traffic record once the kernel's sources changed."""
import json
import os

import pytest

import bench
from paper_1812_05902_gb300 import scenes


def test_ops_per_ray_counts_each_stage():
    fr = scenes.c1(scale=0.001)[0]
    surf = sum(bench.OPS_SURF[s.type] for s in fr.optics.surfaces)
    assert bench.ops_per_ray(fr, 3.0) == bench.OPS_RAY_BASE + surf + 3.0 * bench.OPS_STEP[scenes.RK4]
    fr.optics.mie = scenes.Mie()
    assert bench.ops_per_ray(fr, 3.0) == bench.OPS_RAY_BASE + surf + 3.0 * bench.OPS_STEP[scenes.RK4] + bench.OPS_MIE


def test_optics_variants_copy_per_frame():
    frames = scenes.c1(scale=0.001)
    assert frames[0].optics is frames[1].optics          # the workload shares one camera
    n0 = len(frames[0].optics.surfaces)
    bench.apply_optics_variant(frames, "plenoptic")
    for fr in frames:
        assert len(fr.optics.surfaces) == n0 + 1       # one lenslet array each, not two
        assert fr.optics.surfaces[-1].type == scenes.LENS_ARRAY
    frames = scenes.c1(scale=0.001)
    bench.apply_optics_variant(frames, "mirror")
    assert frames[0].optics.surfaces[0].type == scenes.MIRROR
    assert frames[0].optics.surfaces[0].z < frames[0].optics.aim_z
    frames = scenes.c1(scale=0.001)
    bench.apply_optics_variant(frames, "tilted")
    assert frames[0].optics.sensor_tilt_x != 0.0
    bench.apply_optics_variant(frames, "plain")
    with pytest.raises(SystemExit):
        bench.apply_optics_variant(frames, "fisheye")


def test_roofline_arithmetic():
    fr = scenes.c2(scale=0.1, grid=32)[0]
    steps = 100.0
    rf = bench.roofline([fr], [steps], render_ms=20.0, render_launches=2, sm_max_mhz=2000.0, l1_gbs=30000.0)
    t = 10e-3
    ops = bench.ops_per_ray(fr, steps) * fr.n_rays
    peak = bench.N_SM * bench.ISSUE_LANES_PER_SM * 2000e6 / 1e12
    assert rf["achieved"] == pytest.approx(ops / t / 1e12, rel=1e-3)
    assert rf["peak"] == pytest.approx(peak, rel=1e-3)
    assert rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"], rel=1e-3)
    g = rf["gather"]
    gbytes = bench.GATHER_BYTES_PER_EVAL * bench.EVALS_PER_STEP[scenes.RK4] * steps * fr.n_rays
    assert g["achieved"] == pytest.approx(gbytes / t / 1e9, rel=1e-3)
    assert g["frac_measured"] == pytest.approx(g["achieved"] / 30000.0, rel=1e-3)
    assert bench.roofline([fr], [steps], 20.0, 0, 2000.0) is None


def test_traffic_record_dropped_when_sources_change(tmp_path, monkeypatch):
    rec = {"source_hash": bench.kernel_source_hash("render"), "dram_bytes_read": 10, "dram_bytes_write": 5}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "t.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_1812_05902_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in bench.KERNEL_SOURCES["render"]:
        (csrc / name).write_bytes(open(os.path.join(os.path.dirname(bench.__file__), "paper_1812_05902_gb300",
                                                    "csrc", name), "rb").read())
    assert bench.recorded_traffic("t") == 15
    (csrc / "trace.cuh").write_text("// changed\n")
    assert bench.recorded_traffic("t") is None
    assert bench.recorded_traffic("missing") is None


def test_shard_ranges_cover_the_sources_once():
    for n in (1, 7, 100000):
        for world in (1, 2, 3, 8):
            ranges = [bench.shard_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            assert max(h - l for l, h in ranges) - min(h - l for l, h in ranges) <= 1


def test_oracle_subset_keeps_the_image_rays():
    fr = scenes.c4(scale=0.2, grid=16)[0]
    sub = bench.c4_subset(fr)
    assert len(sub.sources) == 10000 and sub.rays_per_source == 100
    assert sub.sources is not fr.sources or len(fr.sources) == 10000
    assert fr.rays_per_source == 10000                  # the frame itself is untouched
    assert (sub.sources == fr.sources[:10000]).all()


def test_both_arms_print_the_same_config():
    import argparse
    for wl, sur in (("c4", False), ("c1", False), ("c2", True)):
        a = argparse.Namespace(workload=wl, scale=0.01, optics="plain", surrogate=sur, gpus=1)
        assert bench.config_for(a) == bench.config_for(argparse.Namespace(**vars(a)))
        assert bench.config_for(a)["rays_per_step"] > 0
    a = argparse.Namespace(workload="c4", scale=0.01, optics="plain", surrogate=False, gpus=4)
    assert "all-reduce" in bench.config_for(a)["parallelism"]


def test_traffic_record_scaled_to_the_launch(tmp_path, monkeypatch):
    rec = {"source_hash": bench.kernel_source_hash("render"), "dram_bytes_read": 300, "dram_bytes_write": 100,
           "rays_per_launch": 1000, "rays_per_cta": 2048}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "t.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_1812_05902_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in bench.KERNEL_SOURCES["render"]:
        (csrc / name).write_bytes(open(os.path.join(os.path.dirname(bench.__file__), "paper_1812_05902_gb300",
                                                    "csrc", name), "rb").read())
    assert bench.recorded_traffic("t", rays_per_cta=2048, scale_to_rays=5000) == 2000
    assert bench.recorded_traffic("t", rays_per_cta=256, scale_to_rays=5000) is None
    assert bench.recorded_traffic("t") == 400


def test_roofline_of_a_sharded_launch():
    fr = scenes.c2(scale=0.1, grid=32)[0]
    whole = bench.roofline([fr], [100.0], 10.0, 1, 2000.0, l1_gbs=30000.0)
    half = bench.roofline([fr], [100.0], 5.0, 1, 2000.0, l1_gbs=30000.0, ray_frac=0.5)
    assert half["achieved"] == pytest.approx(whole["achieved"], rel=1e-3)
    assert half["rays_per_launch"] == whole["rays_per_launch"] // 2


def test_traffic_record_of_a_fixed_part_is_not_scaled(tmp_path, monkeypatch):
    rec = {"source_hash": bench.kernel_source_hash("render"), "dram_bytes_read": 300, "dram_bytes_write": 100,
           "rays_per_launch": 1000, "scales_with_rays": False}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "t.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_1812_05902_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in bench.KERNEL_SOURCES["render"]:
        (csrc / name).write_bytes(open(os.path.join(os.path.dirname(bench.__file__), "paper_1812_05902_gb300",
                                                    "csrc", name), "rb").read())
    assert bench.recorded_traffic("t", scale_to_rays=5000) == 400
