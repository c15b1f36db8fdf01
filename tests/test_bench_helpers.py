"""CPU checks of bench.py's bookkeeping: the kernel-source hash that keys the recorded DRAM
traffic ignores comments and blank lines but not code, and the recorded capture figures are
read only while their hash matches the sources."""
import os
import shutil

import pytest

import bench

SRC = ("ara_ylt.cu", "ara_device.cuh")


@pytest.fixture()
def tree(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1606_04473_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in SRC:
        shutil.copy(os.path.join(bench.ROOT, "paper_1606_04473_gb300", "csrc", name), csrc / name)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def test_hash_ignores_comments_and_blank_lines(tree):
    h0 = bench.kernel_source_sha()
    f = tree / "paper_1606_04473_gb300" / "csrc" / "ara_ylt.cu"
    text = f.read_text()
    f.write_text("// a new comment line\n\n" + text.replace("\n", "\n\n", 3) + "\n// trailing\n")
    assert bench.kernel_source_sha() == h0
    f.write_text(text.replace("BK_CHUNK_IDS / 32", "BK_CHUNK_IDS / 16", 1))
    assert bench.kernel_source_sha() != h0


def test_profile_figures_are_read_only_for_the_matching_source(tree):
    prof = tree / "profiles" / "k_ylt_bulk_paper_scale.txt"
    prof.write_text(f"# figures\nkernel_source_sha: {bench.kernel_source_sha()}\ndram_bytes_per_event: 4.25\n"
                    "l2_hit_rate_pct: 61.5 (lts__t_sector_hit_rate.pct)\n")
    fig = bench.ncu_profile_figures()
    assert fig["dram_bytes_per_event"] == pytest.approx(4.25)
    assert fig["l2_hit_rate_pct"] == pytest.approx(61.5)
    prof.write_text("kernel_source_sha: 0000000000000000\ndram_bytes_per_event: 4.25\n")
    assert bench.ncu_profile_figures() == {}
