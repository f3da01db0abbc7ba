"""Host logic of bench.py that needs no GPU: the DRAM-traffic figure comes from the
committed ncu table only while the kernel's source is the one that was captured."""
import hashlib
import os

import bench


def _tree(tmp_path, src_text, table_sha):
    csrc = tmp_path / "paper_2105_01028_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text(src_text)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.txt").write_text("# kernel source sha bytes capture\n"
                                      f"my_kernel k.cu {table_sha} 12.5 cap.md\n")


def test_traffic_scales_with_updates_while_the_source_is_unchanged(tmp_path, monkeypatch):
    src = "__global__ void my_kernel() {}\n"
    _tree(tmp_path, src, hashlib.sha256(src.encode()).hexdigest()[:16])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("my_kernel", 1000) == 12500.0
    assert bench.measured_traffic("other_kernel", 1000) is None


def test_traffic_is_withheld_once_the_source_changes(tmp_path, monkeypatch):
    src = "__global__ void my_kernel() {}\n"
    _tree(tmp_path, src, hashlib.sha256(src.encode()).hexdigest()[:16])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "paper_2105_01028_gb300" / "csrc" / "k.cu").write_text(src + "// edited\n")
    assert bench.measured_traffic("my_kernel", 1000) is None


def test_committed_table_names_existing_sources_and_captures():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for ln in open(os.path.join(root, "profiles", "traffic.txt")).read().splitlines():
        if not ln.strip() or ln.startswith("#"):
            continue
        kernel, src, sha, per_update, capture = ln.split()[:5]
        assert os.path.isfile(os.path.join(root, "paper_2105_01028_gb300", "csrc", src)), ln
        assert os.path.isfile(os.path.join(root, "profiles", capture)), ln
        assert len(sha) == 16 and float(per_update) > 0.0


PEAKS = {"hbm_gbs": 6689.5, "bf16_tflops": 1917.3, "bf16_tflops_sustained": 1725.0, "sm_max_mhz": 2070.0,
         "_source": "measured"}


def test_iteration_roofline_follows_arithmetic_intensity():
    """Below the ridge point (compute peak / HBM peak) the iteration kernel is reported on
    the HBM roofline, above it on the compute roofline; both fractions are given."""
    nv, na = 96 * 96 * 64, 192
    kms = [0.45 * 10, 1.03 * 10, 0.06 * 10]  # summed ms of 10 profiled steps
    k, r = bench.kernel_roofline(nv, na, na, kms, 10, 1.7, "bf16", PEAKS)
    s = k[1]
    assert r["kernel"] == "scatter_bf16" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    nbytes = nv * na * 20 + nv * 12
    assert s["algorithmic_bytes"] == nbytes
    assert abs(r["achieved"] - nbytes / 1.03e-3 / 1e9) < 1e-6 * r["achieved"]
    assert abs(s["arithmetic_intensity"] - 2.0 * na * na * nv * 1.7 / nbytes) < 1e-9 * s["arithmetic_intensity"]
    assert s["arithmetic_intensity"] < s["ridge_flop_per_byte"]
    assert abs(s["ridge_flop_per_byte"] - 1725.0e12 / 6689.5e9) < 1e-9
    assert 0.0 < s["compute_frac"] < s["hbm_frac"] == r["frac"]
    # many iterations per voxel: compute-bound, on the sustained BF16 peak
    k, r = bench.kernel_roofline(nv, na, na, [4.5, 40.0, 0.6], 10, 50.0, "bf16", PEAKS)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s" and r["peak"] == 1725.0


def test_fp32_iteration_and_exact_solve_rooflines(monkeypatch):
    monkeypatch.setattr(bench, "sm_count", lambda: 152)
    nv, na = 96 * 96 * 64, 192
    k, r = bench.kernel_roofline(nv, na, na, [4.5, 290.0, 0.6], 10, 12.9, "fp32", PEAKS)
    assert r["bound"] == "alu" and abs(r["peak"] - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9
    assert "FFMA" in r["peak_source"]
    # the exact solve on the tensor cores: one product per voxel, reported on HBM
    k, r = bench.kernel_roofline(nv, na, na, [4.5, 3.05, 0.6], 10, 1.0, "fp32", PEAKS, exact="tc")
    s = k[1]
    assert s["name"] == "exact_tc" and s["bound"] == "hbm" and s["algorithmic_bytes"] == nv * na * 12 + nv * 5
    assert s["tensor_tflops_3xtf32"] > 0
    assert r["kernel"] == "sweep"  # the sweep (0.45 ms) outweighs the product (0.305 ms)
