"""Host-side rules of bench.py (no GPU): default step counts, and the DRAM
traffic of an evaluator launch reported only while the evaluator source is
the one the ncu capture was taken on."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_defaults(monkeypatch):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "kitc"
    assert a.precision == "mixed_leaf"
    assert (a.theta, a.degree, a.leaf, a.mac) == (bench.THETA, bench.DEGREE, bench.LEAF, bench.MAC)


def test_config_names_the_near_field_form():
    import bench
    monkey = type("A", (), dict(theta=0.68, degree=9, leaf=4000, mac="all", literal=False))
    assert "leaf" in bench.config(monkey, "mixed_leaf")["near_differences"]
    assert "hi/lo" in bench.config(monkey, "mixed")["near_differences"]
    assert bench.config(monkey, "fp64 (CPU oracle)")["near_differences"] == "FP64"


def test_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    import hashlib
    import bench
    src = open(os.path.join(ROOT, "paper_1902_02250_gb300", "csrc", "evaluate.cu"), "rb").read()
    rec = {"evaluate_cu_sha256": hashlib.sha256(src).hexdigest(), "dram_bytes_per_launch": 123.0,
           "rotlet": {"dram_bytes_per_launch": 456.0}}
    (tmp_path / "profiles").mkdir()
    json.dump(rec, open(tmp_path / "profiles" / "eval_traffic.json", "w"))
    csrc = tmp_path / "paper_1902_02250_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "evaluate.cu").write_bytes(src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_per_launch() == 123.0
    assert bench.traffic_per_launch("rotlet") == 456.0
    # an evaluator that differs by one byte from the captured one reports no traffic
    (csrc / "evaluate.cu").write_bytes(src + b"\n")
    assert bench.traffic_per_launch() is None and bench.traffic_per_launch("rotlet") is None


def test_committed_traffic_matches_its_source_or_is_withheld():
    import hashlib
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "eval_traffic.json")))
    src = open(os.path.join(ROOT, "paper_1902_02250_gb300", "csrc", "evaluate.cu"), "rb").read()
    if rec["evaluate_cu_sha256"] == hashlib.sha256(src).hexdigest():
        assert bench.traffic_per_launch() == rec["dram_bytes_per_launch"]
    else:
        assert bench.traffic_per_launch() is None
