"""bench.py on the host: the reference arm's JSON line (the CPU oracle) and the
bookkeeping it reports, without a GPU."""
import hashlib
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_prints_the_contract_line():
    bench = load_bench()
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "msbm_n2000_k5_h2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "s/solve" and d["higher_is_better"] is False and d["value"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["config"]["workload"] == "msbm_n2000_k5_h2"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "s/solve", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_recorded_traffic_follows_the_sources(tmp_path, monkeypatch):
    """roofline.traffic is reported only while the kernel's sources hash as recorded."""
    bench = load_bench()
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    sha = hashlib.sha256(b"kernel v1").hexdigest()
    (tmp_path / "profiles" / "s.md").write_text(f"traffic_bytes_per_launch: 1234\nsource_sha256 k.cu: {sha}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("s.md", ["k.cu"]) == 1234
    src.write_text("kernel v2")
    assert bench.recorded_traffic("s.md", ["k.cu"]) is None
    assert bench.recorded_traffic("missing.md", ["k.cu"]) is None


def test_operator_bytes_at_the_bench_workload():
    """The fused operator's algorithmic bytes per launch at m-SBM n = 1M (nnz = 32,006,342,
    BF16 weights, FP32 vectors, block 4): 4 (n + 1) + 6 nnz + 37 n = 233,038,056 bytes."""
    bench = load_bench()
    assert bench.operator_bytes(1_000_000, 32_006_342, 2, 4, 4) == 233_038_056
