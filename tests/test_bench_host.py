"""Host logic of bench.py, on the CPU: the algorithmic SFU accounting of the
roofline, the lookup of the committed ncu traffic and the measured peaks."""
import json
import types

import pytest

import bench


def test_algorithmic_ops_count_sources_and_model_branches():
    st = types.SimpleNamespace(source_evaluations=1000, model_point_steps=50,
                               model_sfu_ex2=170, model_sfu_slow=160,
                               farfield_point_sources=0, farfield_node_evaluations=0)
    slow, ex2 = bench.algorithmic_sfu_ops(st)
    # one 1/R and one exp per point and source, plus the model's own counts
    assert (slow, ex2) == (1160, 1170)
    assert bench.executed_sfu_ops(st) == (1160, 1170)


def test_far_field_pairs_count_as_algorithmic_work_nodes_as_executed():
    """A pair the far field interpolates is work the method requires (the
    superposed source at that point); the kernel executes node evaluations
    instead."""
    st = types.SimpleNamespace(source_evaluations=1000, model_point_steps=50,
                               model_sfu_ex2=170, model_sfu_slow=160,
                               farfield_point_sources=4000, farfield_node_evaluations=250)
    assert bench.algorithmic_sfu_ops(st) == (5160, 5170)
    assert bench.executed_sfu_ops(st) == (1410, 1420)
    rates = {"rsqrt": 16.0, "ex2": 32.0}
    t = bench.sfu_time_s(16.0, 32.0, rates)
    assert t == pytest.approx(2.0 / (bench.SM_COUNT * bench.SM_MAX_MHZ * 1e6))


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


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference times the FP64 oracle on the host cores and
    prints one JSON line with the keys of the bench contract, its e2e equal to
    its value and no host-device traffic."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--workload", "line_4096", "--steps", "2", "--warmup", "1",
                        "--cpu-seconds", "0.2"], cwd=root, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in out, k
    assert out["impl"] == "reference" and out["steps"] == 2 and out["warmup"] == 1
    assert out["value"] > 0 and out["higher_is_better"] is True
    assert out["config"]["workload"] == "line_4096"
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] >= 1
    assert out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"] == {"value": out["value"], "unit": out["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}


def test_profile_summaries_name_their_commands():
    """Each ncu summary under profiles/ gives the command that made it, with
    ncu's clocks left alone (--clock-control none), and runs committed files
    only (nothing under the git-ignored working folder)."""
    import glob
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    files = sorted(glob.glob(os.path.join(root, "profiles", "*.md")))
    assert files
    for f in files:
        text = open(f).read()
        assert "ommand" in text, f
        assert "_work/" not in text, f
        if "ncu " in text:
            assert "--clock-control none" in text, f


@pytest.mark.parametrize("world", [2, 3, 8])
def test_strong_scaling_shards_cover_the_instance_once(world):
    """bench.py --scaling strong: the ranks' shards hold every point of the
    one instance exactly once, with the instance's coordinates (a slab is a
    grid of its own whose k_offset keeps the parent's z; the batch's
    specimens are dealt out whole), and the line divides the whole
    instance's work by the time."""
    import numpy as np
    whole = bench.make_workload("block_256", 0, 1, False)
    g = whole.specimens[0].grid
    zs = []
    for r in range(world):
        w = bench.make_workload("block_256", r, world, True)
        assert w.meta["whole_point_updates"] == whole.point_updates
        sg = w.specimens[0].grid
        assert sg.dims[:2] == g.dims[:2]
        zs.append(sg.coords(np.arange(0, sg.n, sg.dims[0] * sg.dims[1]))[2])
    np.testing.assert_array_equal(np.concatenate(zs),
                                  g.coords(np.arange(0, g.n, g.dims[0] * g.dims[1]))[2])
    batch = bench.make_workload("batch_64", 0, 1, False)
    key = lambda sp: (sp.grid.dims, float(sp.source.t_offset), float(sp.source.tracks[0, 5]))
    got = sorted(key(sp) for r in range(world)
                 for sp in bench.make_workload("batch_64", r, world, True).specimens)
    assert got == sorted(key(sp) for sp in batch.specimens)
