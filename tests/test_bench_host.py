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
