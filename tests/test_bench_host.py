"""Host-side rules of bench.py (no GPU): default step counts, and the DRAM
traffic of an evaluator launch reported only while the evaluator source is
the one the ncu capture was taken on."""
import json
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_defaults(monkeypatch):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "kitc"


def test_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "eval_traffic.json")))
    assert bench.traffic_per_launch() == rec["dram_bytes_per_launch"]
    assert bench.traffic_per_launch("rotlet") == rec["rotlet"]["dram_bytes_per_launch"]
    # a copy of the tree whose evaluator differs by one byte reports no traffic
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(ROOT, "profiles", "eval_traffic.json"), tmp_path / "profiles")
    csrc = tmp_path / "paper_1902_02250_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = open(os.path.join(ROOT, "paper_1902_02250_gb300", "csrc", "evaluate.cu"), "rb").read()
    (csrc / "evaluate.cu").write_bytes(src + b"\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_per_launch() is None and bench.traffic_per_launch("rotlet") is None
    (csrc / "evaluate.cu").write_bytes(src)
    assert bench.traffic_per_launch() == rec["dram_bytes_per_launch"]
