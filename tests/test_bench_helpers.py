"""Host-side helpers of the benchmark (CPU only): the kernel source hash that keys the committed
ncu counters, and the arithmetic of the whole-job figures."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _copy_sources(tmp_path):
    for rel in bench.KERNEL_SOURCES:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), dst)
    return str(tmp_path)


def test_kernel_hash_ignores_comments_but_not_code(tmp_path):
    root = _copy_sources(tmp_path)
    h0 = bench.kernel_sha(root)
    assert h0 == bench.kernel_sha()
    src = tmp_path / bench.KERNEL_SOURCES[0]
    text = src.read_text()
    src.write_text("// a new comment line\n" + text.replace("namespace sgn {", "namespace sgn {  /* inline */", 1) + "\n\n")
    assert bench.kernel_sha(root) == h0
    src.write_text(text + "\nstatic const int kHashProbe = 1;\n")
    assert bench.kernel_sha(root) != h0


def test_committed_counters_match_the_current_kernel():
    c = bench.profiled_counters()
    if not c:
        pytest.skip("the committed ncu counters were taken on other kernel sources (the bench reports them as null)")
    assert c["dram_bytes_per_launch"] > 0 and c["warp_instructions_per_launch"] > 0


def test_single_rank_throughput_and_ms():
    ranks = bench.Ranks("gloo")
    assert ranks.throughput(15_360_000 * 1000, 80.0) == pytest.approx(1.92e11)


def test_issue_and_l1_pipe_rooflines(monkeypatch):
    """The two counter-based rooflines of the bench line: counts of one launch per kernel second
    against one warp instruction per cycle per SM sub-partition, and one L1 data-pipeline wavefront
    per cycle per SM, at the sampled clock (152 SMs at 2070 MHz: 1258.56 and 314.64 G/s)."""
    import types

    import torch

    monkeypatch.setattr(bench, "profiled_counters",
                        lambda: {"warp_instructions_per_launch": 45.0e6, "l1_lsu_wavefronts_per_launch": 15.0e6})
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda dev: types.SimpleNamespace(multi_processor_count=152))
    clk = {"sm_mhz": 2070.0}
    issue = bench.issue_roofline(75e-6, clk, None)
    assert issue["peak"] == pytest.approx(1258.56) and issue["achieved"] == pytest.approx(600.0)
    l1 = bench.l1_pipe_roofline(75e-6, clk, None)
    assert l1["peak"] == pytest.approx(314.64) and l1["achieved"] == pytest.approx(200.0)
    assert l1["frac"] == pytest.approx(200.0 / 314.64)
    monkeypatch.setattr(bench, "profiled_counters", lambda: {})
    assert bench.issue_roofline(75e-6, clk, None) is None and bench.l1_pipe_roofline(75e-6, clk, None) is None
