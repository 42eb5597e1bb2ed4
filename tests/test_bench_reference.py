"""bench.py's reference arm (the oracle on the timed workload) on CPU, through both of its paths
on a small mesh: the whole oracle operator, and the bounded sample it takes on meshes too large
to build whole in a bench run (the operator restricted to one lattice row, the other rows'
products scaled by the partition's product work).  Both print one JSON line with the arm's
metric and a positive rate; the sampled line says what it sampled."""
import io
import json
import os
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(monkeypatch, sample_above):
    monkeypatch.setattr(bench, "REF_SAMPLE_ABOVE", sample_above)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--config", "small", "--steps", "2",
                                      "--warmup", "1"])
    args = bench.parse()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.reference_arm(args)
    lines = [l for l in buf.getvalue().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_whole_and_sampled(monkeypatch):
    whole = _run(monkeypatch, 10 ** 9)
    sampled = _run(monkeypatch, 1000)
    for d in (whole, sampled):
        assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "steps/s"
        assert d["value"] > 0 and d["steps"] == 2 and d["cpu_baseline"]["kind"] == "oracle"
        assert d["e2e"]["h2d_bytes_per_step"] == 0
    assert whole["cpu_baseline"]["rows_sampled"] == whole["config"]["n_elem"]
    assert 0 < sampled["cpu_baseline"]["rows_sampled"] < sampled["config"]["n_elem"]
    assert "lattice row" in sampled["cpu_baseline"]["sample"]
