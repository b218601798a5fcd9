"""Roofline bookkeeping of bench.py (no GPU): algorithmic bytes per site
update, the comment-insensitive kernel source hash and the parsing of the
committed ncu summaries."""
import os

import bench


def test_algorithmic_bytes_per_site():
    """Read + write of every stored value once: 2 (Q s_f + n_b s_b); the
    comparator stores no variance."""
    assert bench.algorithmic_bytes_per_site(3, "f32") == 200
    assert bench.algorithmic_bytes_per_site(2, "f32") == 96
    assert bench.algorithmic_bytes_per_site(2, "f16") == 60
    assert bench.algorithmic_bytes_per_site(2, "bf16") == 60
    assert bench.algorithmic_bytes_per_site(1, "f64") == 64
    assert bench.algorithmic_bytes_per_site(3, "f32", "standard") == 152


def test_code_only_ignores_comments_not_code():
    a = "int x = 1; // note\n/* block\n comment */ int y = 2;\n"
    b = "int x = 1;\n int y = 2;   // other words\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only('s = "// not a comment";') != bench._code_only("s = ;")
    assert bench._code_only("int x = 1;") != bench._code_only("int x = 2;")


def test_kernel_hashes_cover_their_own_sources():
    assert bench.kernel_source_hash() != bench.kernel_source_hash("std_step_kernel")
    assert bench.kernel_source_hash("step_fast_kernel") == bench.kernel_source_hash()
    for files in [bench.KERNEL_SOURCES, *bench.KERNEL_SOURCES_BY_KERNEL.values()]:
        for f in files:
            assert os.path.exists(os.path.join(bench.ROOT, "paper_2501_00620_gb300", "csrc", f))


def test_profiled_traffic_needs_the_current_source(tmp_path, monkeypatch):
    """A summary's DRAM bytes count only if its kernel_source_sha is the hash
    of the kernel's current code."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "std_step_kernel_std3d_f32.md").write_text(
        "# summary\n\n- kernel_source_sha: `aaaa`\n- dram_bytes_per_launch: 123456\n")
    (prof / "step_fast_kernel_turb3d_f32.md").write_text(
        "- kernel_source_sha: `bbbb`\n- dram_bytes_per_launch: 99\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kernel=None: "aaaa")
    assert bench.profiled_traffic("std_step_kernel", "std3d", "f32") == 123456.0
    assert bench.profiled_traffic("step_fast_kernel", "turb3d", "f32") is None
    assert bench.profiled_traffic("nosuch_kernel", "turb3d", "f32") is None
