"""Host logic of bench.py: the traffic record is keyed on the step-kernel sources without
their comments (a comment edit keeps the counters valid, a code edit invalidates them)."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    b = _bench()
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    f = tmp_path / "k.cu"
    f.write_text("int a = 1;  // one\n\n// note\nint b = 2;\n")
    h0 = b.kernel_source_hash(["k.cu"])
    f.write_text("int a = 1;  // first\n// another note\n\nint b = 2;   \n")
    assert b.kernel_source_hash(["k.cu"]) == h0
    f.write_text("int a = 1;\nint b = 3;\n")
    assert b.kernel_source_hash(["k.cu"]) != h0


def test_traffic_record_scales_per_node(tmp_path, monkeypatch):
    b = _bench()
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_text("int a;\n")
    rec = {"nodes": 100, "dram_bytes_per_launch": 7200.0, "sources": ["k.cu"],
           "source_sha256": b.kernel_source_hash(["k.cu"])}
    (tmp_path / "profiles" / "step_kernel_traffic.json").write_text(json.dumps(rec))
    assert b.step_kernel_traffic(400) == 4 * 7200.0
    (tmp_path / "k.cu").write_text("int a, b;\n")           # the kernel changed: no traffic
    assert b.step_kernel_traffic(400) is None


def test_committed_traffic_record_is_current_and_not_below_the_algorithmic_bytes():
    # the record that bench.py reports as roofline.traffic was captured on the step kernel as
    # committed (same sources), at the benchmark's own size, and it carries at least the 72
    # bytes per node the kernel must move (reads and writes of nine FP32 deviations)
    b = _bench()
    with open(os.path.join(ROOT, "profiles", "step_kernel_traffic.json")) as fh:
        rec = json.load(fh)
    assert b.kernel_source_hash(rec["sources"]) == rec["source_sha256"]
    assert rec["nodes"] == 4096 * 4096
    t = b.step_kernel_traffic(rec["nodes"])
    assert t is not None and t >= 72 * rec["nodes"]
    reads = sum(x[0] for x in rec["launches"]) / len(rec["launches"])
    writes = sum(x[1] for x in rec["launches"]) / len(rec["launches"])
    assert reads >= 36 * rec["nodes"] and writes >= 36 * rec["nodes"]
