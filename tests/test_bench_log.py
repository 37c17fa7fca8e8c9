"""bench.py's result line: printed once on stdout and, with --jsonl, appended
as one record per run to a JSON-lines file (host logic, no GPU)."""

import argparse
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_emit_prints_one_line_and_appends_records(tmp_path, capsys):
    bench = _bench()
    log = tmp_path / "runs.jsonl"
    a = argparse.Namespace(jsonl=str(log))
    bench.emit({"metric": "m", "value": 1.5}, a)
    bench.emit({"metric": "m", "value": 2.5}, a)
    out = capsys.readouterr().out.strip().splitlines()
    assert [json.loads(x)["value"] for x in out] == [1.5, 2.5]
    recs = [json.loads(x) for x in log.read_text().splitlines()]
    assert [r["value"] for r in recs] == [1.5, 2.5]


def test_emit_without_log_only_prints(capsys):
    bench = _bench()
    bench.emit({"value": 3.0}, argparse.Namespace(jsonl=None))
    assert json.loads(capsys.readouterr().out)["value"] == 3.0
