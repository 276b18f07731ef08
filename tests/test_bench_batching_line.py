"""The default bench line's batching object, on the CPU: the child run's JSON
line is reduced to the fields the plain line carries, and a child that fails,
prints nothing or runs out of time yields an error entry instead of breaking
the plain line.  subprocess.run is replaced by a fake; no GPU is involved."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

CHILD_LINE = {
    "metric": bench.METRIC, "value": 19306.3, "unit": "rows/s", "ms_per_step": 424.3, "steps": 2, "warmup": 3,
    "config": {"workload": bench.WORKLOADS["batching"]["desc"], "row_iters_mean": 63.2, "row_iters_max": 300},
    "schedule": {"code": 1, "autotuned": True, "cuda_graph": True},
    "fidelity": {"mean": 0.99819, "frac_ge_0.99": 0.99744},
    "roofline": {"kernel": "k_solver", "achieved": 2.4, "peak": 80.5, "unit": "TFLOP/s", "frac": 0.0299,
                 "solver_ms": 419.5, "traffic": None},
    "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []},
    "gpu_launches": 10,
}


class _Done:
    def __init__(self, rc, out, err=""):
        self.returncode, self.stdout, self.stderr = rc, out, err


def test_child_line_is_reduced_to_the_carried_fields(monkeypatch):
    seen = {}

    def fake_run(cmd, **kw):
        seen["cmd"], seen["env"] = cmd, kw.get("env", {})
        return _Done(0, "warming up\n" + json.dumps(CHILD_LINE) + "\n")

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr(subprocess, "run", fake_run)
    got = bench.batching_child_line()
    assert "--workload" in seen["cmd"] and seen["cmd"][seen["cmd"].index("--workload") + 1] == "batching"
    assert "--no-arms" in seen["cmd"] and "--no-sweep" in seen["cmd"]  # the child never starts another child
    assert "RANK" not in seen["env"]
    assert got["value"] == CHILD_LINE["value"] and got["unit"] == "rows/s"
    assert got["workload"] == bench.WORKLOADS["batching"]["desc"]
    assert got["row_iters_mean"] == 63.2 and got["schedule"]["code"] == 1
    assert got["roofline"]["frac"] == CHILD_LINE["roofline"]["frac"]
    assert "traffic" not in got["roofline"] and "metric" not in got


def test_failing_silent_or_slow_children_give_an_error_entry(monkeypatch):
    monkeypatch.setattr(subprocess, "run", lambda cmd, **kw: _Done(1, "", "Traceback ... CUDA error"))
    assert "error" in bench.batching_child_line()
    monkeypatch.setattr(subprocess, "run", lambda cmd, **kw: _Done(0, "no json here\n"))
    assert "error" in bench.batching_child_line()

    def slow(cmd, **kw):
        raise subprocess.TimeoutExpired(cmd, kw.get("timeout"))

    monkeypatch.setattr(subprocess, "run", slow)
    assert "TimeoutExpired" in bench.batching_child_line(timeout_s=1.0)["error"]
