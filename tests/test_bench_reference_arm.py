"""bench.py's reference arm (the oracle timed on the host cores) prints one JSON line
with the contract's keys; run on the smallest workload (P2 on 8^3 cubes)."""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_line_p2_n8(monkeypatch, capsys):
    import bench

    wl, cfg = bench.SINGLE["p2_n8"]
    monkeypatch.setattr(bench, "WORKLOAD", wl)
    monkeypatch.setattr(bench, "CONFIG", cfg)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    bench.reference_arm(argparse.Namespace(steps=2, warmup=1, gpus=1, workload="p2_n8"))
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["config"]["n_h"] == 3375
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
