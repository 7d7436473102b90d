"""The benchmark's reference arm (the CPU oracle, no GPU) prints one JSON line with the keys the
benchmark contract asks for, on the small fingertip-press workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "fingertip_press", "--steps", "1", "--warmup", "0", "--cpu-seconds", "2"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "steps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1
    assert d["config"]["workload"].startswith("fingertip_press")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_pcg_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    """The roofline's `traffic` comes from the committed ncu summary only while pcg.cu is the source that
    was captured; any other source gives null."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "paper_2609_25653_b300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (src / "pcg.cu").write_text("// captured source\n")
    sha = hashlib.sha256(b"// captured source\n").hexdigest()[:16]
    rec = {"captures": [{"kernel": "k_pcg", "workload": "w", "pcg_cu_sha16": sha, "dram_bytes_per_launch": 123}]}
    (tmp_path / "profiles" / "pcg_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.pcg_traffic("k_pcg", "w") == 123
    assert bench.pcg_traffic("k_pcg32", "w") is None        # other kernel
    assert bench.pcg_traffic("k_pcg", "other") is None      # other workload
    (src / "pcg.cu").write_text("// changed source\n")
    assert bench.pcg_traffic("k_pcg", "w") is None          # changed since the capture
