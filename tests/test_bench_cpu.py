"""bench.py host logic on the CPU: the reference arm's JSON line (the FP64
oracle timed on a bounded sample) and the workload descriptions."""
import argparse
import json

import bench


def test_reference_arm_prints_the_contract_line(capsys):
    args = argparse.Namespace(workload="2d_n127_M3_fp64", steps=1, warmup=3, gpus=1)
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "impl", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == line["unit"] == "DOF-sweeps/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["config"]["workload"] == "2d_n127_M3_fp64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and "127^2" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "DOF-sweeps/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(argparse.Namespace(workload="3d_n255_M5_fp64", steps=1, warmup=3, gpus=2))
    assert capsys.readouterr().out == ""


def test_every_workload_describes_itself():
    for name, w in bench.workloads().items():
        cfg = bench.config_of(w)
        assert cfg["workload"] == name and cfg["dofs"] == w.n ** w.ndim
        assert cfg["nodes"] in ("gauss-lobatto", "gauss-radau-right", "gauss-legendre")
        assert "L2" in cfg["l2"]
