"""Host logic of bench.py, on the CPU: the algorithmic SFU accounting of the
roofline, the lookup of the committed ncu traffic and the measured peaks."""
import json
import types

import pytest

import bench


def test_algorithmic_ops_count_sources_and_model_branches():
    st = types.SimpleNamespace(source_evaluations=1000, model_point_steps=50,
                               model_sfu_ex2=170, model_sfu_slow=160)
    slow, ex2 = bench.algorithmic_sfu_ops(st)
    # one 1/R and one exp per point and source, plus the model's own counts
    assert (slow, ex2) == (1160, 1170)


def test_traffic_only_for_the_captured_kernel_workload_and_steps(tmp_path, monkeypatch):
    summary = {"kernel_source_hash": bench.kernel_source_hash(), "workload": "block_256",
               "dram_bytes_per_launch_by_steps": {"128": 111, "256": 222}}
    path = tmp_path / "summary.json"
    path.write_text(json.dumps(summary))
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(path))
    assert bench.ncu_traffic("block_256", 128)[0] == 111
    assert bench.ncu_traffic("block_256", 256)[0] == 222
    assert bench.ncu_traffic("block_256", 64)[0] is None
    assert bench.ncu_traffic("part_512", 128)[0] is None
    summary["kernel_source_hash"] = "0" * 16
    path.write_text(json.dumps(summary))
    assert bench.ncu_traffic("block_256", 128)[0] is None


def test_committed_traffic_matches_the_committed_kernel():
    """The committed ncu summary was taken on the committed kernel source, so
    the bench line reports its traffic."""
    assert bench.ncu_traffic("block_256", 128)[0] is not None


def test_measured_hbm_peak(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_hbm_gbs(default=1.0) == 1.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6500.0}))
    assert bench.measured_hbm_gbs(default=1.0) == pytest.approx(6500.0)
