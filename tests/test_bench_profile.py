"""The benchmark reads the DRAM traffic of the streaming propose from the
committed ncu summary only while the kernel sources hash to the value the
summary records (CPU)."""

import os

import bench

CSRC = os.path.join(bench.ROOT, "paper_1206_6409_gb300", "csrc")
SRCS = [os.path.join(CSRC, f) for f in ("kernels_propose.cu", "propose_plan.cu")]


def test_committed_summary_matches_the_kernel_sources():
    traffic, src_hash = bench.recorded_traffic(SRCS, "f32")
    assert traffic is not None, f"profiles/propose_all_config2_f32.md was taken on other sources than {src_hash}"
    # DRAM bytes per launch: below the algorithmic X stream (16-bit slab rows), above half of it
    assert 0.8e9 < traffic < 1.7e9


def test_changed_sources_give_no_traffic(tmp_path):
    other = tmp_path / "k.cu"
    other.write_text("// another kernel\n")
    traffic, src_hash = bench.recorded_traffic([str(other)], "f32")
    assert traffic is None and len(src_hash) == 16


def test_missing_summary_gives_no_traffic():
    traffic, _ = bench.recorded_traffic(SRCS, "no-such-mode")
    assert traffic is None
