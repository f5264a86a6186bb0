"""bench.py's reference arm (the oracle timed on the host cores) prints one JSON line
with the contract's keys; run on the two small workloads (P2 on 8^3 cubes, and the
P3 24^3 problem of the differentiable workload)."""
import argparse
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.mark.parametrize("workload", ["p2_n8", "p3_n24_adjoint"])
def test_reference_arm_line(monkeypatch, capsys, workload):
    import bench

    wl, cfg = bench.SINGLE[workload] if workload in bench.SINGLE else (bench.ADJOINT, bench.CONFIG_ADJOINT)
    monkeypatch.setattr(bench, "WORKLOAD", wl)
    monkeypatch.setattr(bench, "CONFIG", cfg)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    bench.reference_arm(argparse.Namespace(steps=2, warmup=1, gpus=1, workload=workload))
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["config"]["n_h"] == cfg["n_h"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
