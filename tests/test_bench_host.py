"""Host logic of bench.py: the strips the CPU baseline cuts a workload
into, the kernel a timed region is attributed to, and the config both arms
of the comparison print."""
import os

import numpy as np

import bench
import workloads as wl


def test_strips_cover_the_lattice_once_and_keep_the_body_once():
    p = wl.oscillating_disk()
    for n in (1, 3, 7, 16, 100):
        strips = bench.strip_problems(p, n)
        assert len(strips) == n
        assert sum(q["ny"] for q in strips) == p["ny"]
        assert all(q["nx"] == p["nx"] and q["ny"] >= 1 for q in strips)
        with_body = [q for q in strips if q["body"] is not None]
        assert len(with_body) == 1
        # the body sits at the same place relative to its strip
        lo = 0
        for q in strips:
            if q["body"] is not None:
                assert q["body"]["y"] == p["body"]["y"] - lo
                assert 0 <= q["body"]["y"] < q["ny"]
                assert q["body"]["x"] == p["body"]["x"]
            lo += q["ny"]
        for q in strips:   # the cut edges are walls; west and east as the workload
            assert q["bc"]["south"]["kind"] == q["bc"]["north"]["kind"] == "noslip"
            assert q["bc"]["west"] == p["bc"]["west"] and q["bc"]["east"] == p["bc"]["east"]


def test_strips_keep_the_outer_walls_where_they_reach_them():
    # the paper's cylinder has symmetry walls south and north: the first
    # strip keeps the south one, the last the north one, the cuts are no-slip;
    # a periodic edge becomes a wall unless the strip is the whole lattice
    p = wl.paper_oscillating_cylinder()
    strips = bench.strip_problems(p, 4)
    kinds = [(q["bc"]["south"]["kind"], q["bc"]["north"]["kind"]) for q in strips]
    assert kinds[0] == (p["bc"]["south"]["kind"], "noslip") and kinds[-1] == ("noslip", p["bc"]["north"]["kind"])
    assert all(k == ("noslip", "noslip") for k in kinds[1:-1])
    assert bench.strip_problems(p, 1)[0]["bc"] == p["bc"]
    box = wl.periodic_box(40, 30)
    assert [q["bc"]["south"]["kind"] for q in bench.strip_problems(box, 3)] == ["noslip"] * 3
    assert bench.strip_problems(box, 1)[0]["bc"]["south"]["kind"] == "periodic"


def test_strips_cut_wall_profiles_and_keep_every_body_once():
    # a per-row inlet profile is cut with the rows; several bodies each stay
    # in the one strip that holds its centre
    p = wl.channel_fixed_disk()
    prof = p["bc"]["west"]["ux_profile"]
    for n in (1, 5, 16):
        strips = bench.strip_problems(p, n)
        assert all(len(q["bc"]["west"]["ux_profile"]) == q["ny"] for q in strips)
        assert np.array_equal(np.concatenate([q["bc"]["west"]["ux_profile"] for q in strips]), prof)
    band = bench.row_band(p, 40)
    assert band["ny"] == 40 and len(band["bc"]["west"]["ux_profile"]) == 40
    lo = int(round(p["body"]["y"] - 20))
    assert np.array_equal(band["bc"]["west"]["ux_profile"], prof[lo:lo + 40])
    m = wl.several_bodies()
    strips = bench.strip_problems(m, 16)
    kept = sorted((c["x"], c["y"] + sum(q["ny"] for q in strips[:k]))
                  for k, q in enumerate(strips) for c in q.get("bodies") or [])
    assert kept == sorted((c["x"], c["y"]) for c in m["bodies"])
    for q in strips:
        assert all(0 <= c["y"] < q["ny"] for c in q.get("bodies") or [])


def test_reference_arm_prints_the_contract_line_on_the_host():
    # the reference arm (the oracle on the host cores) on a small workload:
    # one JSON line with the keys the comparison reads
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3",
                        "--workload", "channel_256x128"], cwd=bench.ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "channel_fixed_disk_256x128"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_dominant_kernel_follows_the_node_updates_of_the_region():
    two = {"one_step": 0, "two_step": 10, "lookahead": 1, "tma": 0}
    assert bench.dominant_kernel("f32", ("fused2", 256, 1), two) == "vp_mrt_step2<1, 0, 0>"
    # 3 single steps against 2 two-step launches (4 steps): still the two-step kernel
    mixed = {"one_step": 3, "two_step": 2, "lookahead": 1, "tma": 0}
    assert bench.dominant_kernel("f32", ("fused2", 256, 1), mixed) == "vp_mrt_step2<1, 0, 0>"
    single = {"one_step": 5, "two_step": 2, "lookahead": 1, "tma": 0}
    assert bench.dominant_kernel("f32", ("fused2", 256, 1), single) == "vp_mrt_step<1, 6, 0, 0>"
    assert bench.dominant_kernel("f64", ("scalar", 32, 4), {"one_step": 20}) == "vp_mrt_step<0, 4, 0, 0>"
    assert bench.dominant_kernel("f16", ("pair", 32, 8), {"one_step": 20}) == "vp_mrt_step_pair<2, 5, 0>"
    assert bench.dominant_kernel("f32", ("pair", 32, 8), {"one_step": 20}) == "vp_mrt_step_pair<1, 5, 0>"
    assert bench.dominant_kernel("f32", ("tma", 256, 1), {"tma": 20}) == "vp_mrt_step_tma<1>"


def test_both_arms_print_the_same_config():
    p = wl.oscillating_disk()
    a = bench.bench_config(p, "f32", 1)
    assert a == bench.bench_config(p, "f32", 1)
    assert a["workload"] == "oscillating_disk_2048x1024" and a["storage"] == "f32 deviation"
    assert "151 MB" in a["l2"]   # 72 bytes per node update over 2 097 152 nodes


def test_profiled_traffic_needs_a_matching_source_hash(tmp_path, monkeypatch):
    k = "vp_mrt_step2<1, 0, 0>"
    monkeypatch.setattr(bench, "PROFILE_DIR", str(tmp_path))
    stem = "vp_mrt_step2_1_0_0_w"
    (tmp_path / f"{stem}.md").write_text(f"dram_bytes_per_launch_full_size: 1.5e+08\n"
                                         f"kernel_source_sha256_16: {bench.kernel_source_hash(k)}\n")
    assert bench.profiled_traffic(k, "w") == 1.5e8
    (tmp_path / f"{stem}.md").write_text("dram_bytes_per_launch_full_size: 1.5e+08\n"
                                         "kernel_source_sha256_16: 0000000000000000\n")
    assert bench.profiled_traffic(k, "w") is None


def test_source_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    import shutil
    k = "vp_mrt_step2<"
    (tmp_path / "include").mkdir()
    csrc = tmp_path / "csrc"
    csrc.mkdir()
    shutil.copy(os.path.join(bench.ROOT, "include", "vplbm.h"), tmp_path / "include" / "vplbm.h")
    for f in bench.KERNEL_SOURCES[k]:
        shutil.copy(os.path.join(bench.CSRC, f), csrc / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "CSRC", str(csrc))
    h0 = bench.kernel_source_hash(k)
    src = csrc / "step_fused2.cu"
    text = src.read_text()
    src.write_text(text + "\n// a comment\n/* and a block\n   comment */\n")
    assert bench.kernel_source_hash(k) == h0
    src.write_text(text + "\nstatic int extra_symbol = 1;\n")
    assert bench.kernel_source_hash(k) != h0


def test_reference_band_keeps_the_body_and_walls_the_cut_edges():
    p = bench.workload("oscillating_2048x1024")
    q = bench.row_band(p, 64)
    assert q["nx"] == p["nx"] and q["ny"] == 64
    assert q["bc"]["west"] == p["bc"]["west"] and q["bc"]["east"] == p["bc"]["east"]
    assert q["bc"]["south"]["kind"] == "noslip" and q["bc"]["north"]["kind"] == "noslip"
    assert q["body"] is not None and 0 <= q["body"]["y"] < 64
    assert abs(q["body"]["y"] - 32) <= 1 and q["body"]["x"] == p["body"]["x"]
    assert bench.row_band(p, p["ny"])["body"]["y"] == p["body"]["y"]
