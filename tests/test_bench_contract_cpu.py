"""The reference arm of bench.py (the oracle timed on the host cores) prints one JSON line
with the keys the measurement contract asks for.  Run on a small problem in place of the
128^3 workload so the check takes seconds; the arm's code path is otherwise the one the
full run takes."""
import io
import json
import sys
from contextlib import redirect_stdout

import pase_inputs as pin


def test_reference_arm_json_line(monkeypatch):
    import bench
    pb = pin.build_problem(3, 8, 4, mg_min=4)
    monkeypatch.setattr(bench, "build_workload", lambda nfine=bench.NFINE: (pb, 8))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    out = io.StringIO()
    with redirect_stdout(out):
        rc = bench.main()
    assert rc == 0
    lines = [ln for ln in out.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["warmup"] >= 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == bench.WORKLOAD and line["metric"] == bench.METRIC
