"""bench.py --impl reference runs on the host cores alone: its JSON line keeps
the contract (metric, value, unit, e2e with zero copies, cpu_baseline)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "dofs/s to rel. residual 1e-8"
    assert line["unit"] == "dofs/s" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["config"]["iterations"] > 0


def test_measured_traffic_follows_its_sources(tmp_path, monkeypatch):
    # the bench reports the committed ncu traffic only while every source it
    # names (the sweep kernels, the tile schedule) is the one measured
    sys.path.insert(0, ROOT)
    import bench
    (tmp_path / "profiles").mkdir()
    (tmp_path / "a.cu").write_bytes(b"kernel\n")
    (tmp_path / "b.cpp").write_bytes(b"schedule\n")
    blob = lambda b: __import__("hashlib").sha1(b"blob %d\0" % len(b) + b).hexdigest()
    rec = {"kernel": "aux_gs", "workload": "graded2049", "traffic_bytes_per_launch": 123.0,
           "sources": {"a.cu": blob(b"kernel\n"), "b.cpp": blob(b"schedule\n")}}
    (tmp_path / "profiles" / "roofline_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._measured_traffic("aux_gs", "graded2049") == 123.0
    assert bench._measured_traffic("aux_gs", "kuhn129") is None
    assert bench._measured_traffic("fine_gs", "graded2049") is None
    (tmp_path / "b.cpp").write_bytes(b"schedule changed\n")
    assert bench._measured_traffic("aux_gs", "graded2049") is None
