"""The bench's roofline line reports the DRAM traffic of its dominant kernel only
while the sources that define that kernel hash as they did when the ncu counters
were taken; a record for another kernel class, an edited source or a missing file
gives null.  The committed records resolve against the committed sources."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _with_records(monkeypatch, tmp_path, records):
    import bench
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(records))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(path))
    return bench


def test_record_reported_while_sources_match(monkeypatch, tmp_path):
    import bench
    src = ["bench.py"]
    rec = {"w": {"class": "mg_smooth", "dram_bytes_per_launch": 123, "sources": src,
                 "sources_sha256": bench.sources_sha256(src)}}
    b = _with_records(monkeypatch, tmp_path, rec)
    assert b.captured_traffic("w", "mg_smooth")["dram_bytes_per_launch"] == 123
    assert b.captured_traffic("w", "spmv") is None          # another kernel class
    assert b.captured_traffic("other", "mg_smooth") is None  # no record


def test_record_dropped_when_sources_change(monkeypatch, tmp_path):
    import bench
    f = tmp_path / "kernel.cu"
    f.write_text("__global__ void k() {}\n")
    rel = os.path.relpath(str(f), ROOT)
    rec = {"w": {"class": "mg_smooth", "dram_bytes_per_launch": 1, "sources": [rel],
                 "sources_sha256": bench.sources_sha256([rel])}}
    b = _with_records(monkeypatch, tmp_path, rec)
    assert b.captured_traffic("w", "mg_smooth") is not None
    f.write_text("__global__ void k() { /* changed */ }\n")
    assert b.captured_traffic("w", "mg_smooth") is None
    f.unlink()
    assert b.captured_traffic("w", "mg_smooth") is None


def test_committed_records_resolve():
    import bench
    with open(bench.TRAFFIC_FILE) as fh:
        records = json.load(fh)
    for workload, rec in records.items():
        assert rec["dram_bytes_per_launch"] > 0
        assert os.path.exists(os.path.join(ROOT, rec["summary"])), rec["summary"]
        for src in rec.get("sources", bench.SOLVER_SOURCES):
            assert os.path.exists(os.path.join(ROOT, src)), src


def test_step_model_bytes():
    """The whole-step model: per cell, the stage sweeps (32 + 14 d + d^2) w_s, 11 w_s
    per Helmholtz iteration, (d + 12) 8 + c (5 d + 18) w_s per MG-PCG iteration."""
    import bench
    its = {"p": 15, "T": 10, "w": 10}
    c2 = {"geom": 0, "n": (1, 1, 1), "precision": 0}
    b2 = bench.step_model_bytes(c2, dict(its, u=20))          # two velocity components
    assert abs(b2 - (64 * 8 + 40 * 88 + 15 * (14 * 8 + 4.0 / 3.0 * 28 * 8))) < 1e-9
    assert 10100 < b2 < 10300                                # ~10.2 kB per cell-step
    c3 = {"geom": 1, "n": (1, 1, 1), "precision": 0}
    b3 = bench.step_model_bytes(c3, dict(its, u=30))
    assert 11300 < b3 < 11500                                # ~11.4 kB per cell-step
    mixed = bench.step_model_bytes(dict(c3, precision=1), dict(its, u=30))
    assert mixed < b3                                        # FP32 stencil words
    big = bench.step_model_bytes(dict(c2, n=(256, 512, 1)), dict(its, u=20))
    assert abs(big - b2 * 256 * 512) < 1e-3 * big            # per cell times the cells
