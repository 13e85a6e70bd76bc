"""bench.py host logic on the CPU: the reference arm's JSON line (the FP64
oracle timed on a bounded sample of the workload's own grid), the workload
descriptions and the latency-bound roofline record."""
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
    import oracle as O
    with O.all_cores():
        threads = O.threads()
    assert cb["kind"] == "oracle" and cb["cores"] == threads and cb["value"] == line["value"]
    assert "127^2" in cb["sample"] and line["config"]["n"] == 127
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


def test_latency_record_reports_time_and_launches_per_sweep():
    r = bench.latency_record({}, {"bottom": 0.5}, "bottom", elapsed=0.01, sweeps_total=50, launches=2350)
    assert r["bound"] == "latency" and r["unit"] == "us/sweep"
    assert abs(r["achieved"] - 200.0) < 1e-9 and abs(r["launches_per_sweep"] - 47.0) < 1e-12
    assert r["peak"] is None and r["frac"] is None


def test_alu_roofline_uses_the_measured_fp64_peak():
    prof = {"smooth_fine": {"launches": 10, "total_ms": 1.0, "bytes": 1e9, "fp64_ops": 4e10, "fp32_ops": 0.0}}
    peak = {"ops_per_s": 0.6e12}
    r = bench.roofline(prof, "smooth_fine", "none", {"smooth_fine": 1.0}, peak)
    assert r["bound"] == "alu" and abs(r["peak"] - 0.6) < 1e-12 and "measured" in r["peak_source"]
    assert abs(r["achieved"] - 4e9 / 1e-4 / 1e12) < 1e-9
