"""Host-side helpers of bench.py (no GPU): the recorded DRAM traffic is used
only while the kernel sources match the hash in the profile."""

import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _srcs(root):
    csrc = os.path.join(root, "paper_1206_6409_gb300", "csrc")
    return [os.path.join(csrc, f) for f in ("kernels_propose.cu", "propose_plan.cu")]


def test_recorded_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    import bench

    profile = os.path.join(ROOT, "profiles", "propose_all_config2_f32.md")
    if not os.path.exists(profile):
        pytest.skip("no recorded profile")
    recorded = dict(line.split(":", 1) for line in open(profile)
                    if line.startswith(("dram_bytes_per_launch", "source_sha256")))
    traffic, h = bench.recorded_traffic(_srcs(ROOT), "f32")
    assert len(h) == 16
    if h == recorded["source_sha256"].strip():  # the profile was taken on these sources
        assert traffic == float(recorded["dram_bytes_per_launch"])
    else:
        assert traffic is None
    # a changed kernel source invalidates the record
    changed = tmp_path / "kernels_propose.cu"
    shutil.copy(_srcs(ROOT)[0], changed)
    with open(changed, "a") as f:
        f.write("\n// changed\n")
    traffic2, h2 = bench.recorded_traffic([str(changed), _srcs(ROOT)[1]], "f32")
    assert traffic2 is None and h2 != h
    # no profile for a mode: no traffic
    assert bench.recorded_traffic(_srcs(ROOT), "f64")[0] is None


def test_algorithmic_bytes_per_storage_mode():
    import bench

    assert bench.VALUE_BYTES == {"f64": 8, "f32": 4, "bf16": 2, "binary": 0}
