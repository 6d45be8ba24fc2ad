"""Host logic of bench.py (no GPU): the figures it takes from the committed ncu
summaries are used only while they were captured on the current kernel
source, the FP64 ALU roofline arithmetic, and the DRAM-sector node count of
a porous geometry."""
import numpy as np

import bench


def test_profiled_values_follow_the_kernel_source(tmp_path, monkeypatch):
    h = bench.kernel_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    (tmp_path / "cur.md").write_text("dram_bytes_per_launch: 1.5e+09\nfp64_thread_instructions_per_node: 64.0\n"
                                     "kernel_source_sha256_16: %s\n" % h)
    (tmp_path / "old.md").write_text("dram_bytes_per_launch: 1.5e+09\nkernel_source_sha256_16: 0123456789abcdef\n")
    monkeypatch.setattr(bench, "PROFILE_DIR", str(tmp_path))
    assert bench.profiled_traffic("cur") == 1.5e9
    assert bench.profiled_value("cur", "fp64_thread_instructions_per_node") == 64.0
    assert bench.profiled_traffic("old") is None          # captured on another source
    assert bench.profiled_traffic("missing") is None
    assert bench.profiled_value("cur", "no_such_key") is None


def test_fp64_alu_roofline_arithmetic(tmp_path, monkeypatch):
    (tmp_path / "step_f64_dense_two_lattice_taylor_green_2048.md").write_text(
        "fp64_thread_instructions_per_node: 64.0\nkernel_source_sha256_16: %s\n" % bench.kernel_hash())
    monkeypatch.setattr(bench, "PROFILE_DIR", str(tmp_path))
    r = bench.fp64_alu_roofline(8.0, 152)
    peak = 2 * 152 * 2070e6
    assert r["bound"] == "alu" and r["peak_fp64_inst_per_s"] == peak
    assert abs(r["GLUPS_ceiling"] - peak / 64.0 / 1e9) < 1e-3
    assert abs(r["frac"] - 8.0 / (peak / 64.0 / 1e9)) < 1e-4


def test_sector_nodes_by_brute_force():
    rng = np.random.default_rng(5)
    solid = (rng.random((7, 64)) < 0.6).astype(np.uint8)
    for prec, seg in (("f32", 8), ("f64", 4), ("f16s", 16)):
        want = 0
        for y in range(7):
            for x0 in range(0, 64, seg):
                if (solid[y, x0:x0 + seg] == 0).any():
                    want += seg
        assert bench.sector_nodes(solid, prec) == want


def test_sector_nodes_of_a_box_by_brute_force():
    """The 3-D rows count sectors on the box's rows (z, y) stacked along x."""
    rng = np.random.default_rng(6)
    solid = (rng.random((5, 7, 64)) < 0.6).astype(np.uint8)
    want = 0
    for z in range(5):
        for y in range(7):
            for x0 in range(0, 64, 8):
                if (solid[z, y, x0:x0 + 8] == 0).any():
                    want += 8
    assert bench.sector_nodes(solid.reshape(-1, 64), "f32") == want
