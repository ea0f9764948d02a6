"""bench.py's host-side contract, on the CPU: the reference arm (the oracle on a bounded sample)
prints one JSON line with the required keys, the algorithmic-operation count follows its per-unit
figures, and the committed ncu traffic is used only while the kernel sources it was taken from are
unchanged."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

REQUIRED = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
            "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config")


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3", "--ref-paths", "2048"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in REQUIRED:
        assert k in d, k
    assert d["impl"] == "reference" and d["warmup"] >= 3 and d["value"] > 0
    assert d["config"]["workload"] and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_algorithmic_ops_per_unit():
    c = {"steps": 10, "events": 3, "connections": 2, "connect_steps": 8, "cell_walks": 5}
    want = (10 * bench.OPS_STEP + 3 * bench.OPS_EVENT + 2 * bench.OPS_CONNECT
            + 8 * bench.OPS_CONNECT_STEP + 5 * bench.OPS_CELL_WALK)
    assert bench.algorithmic_ops(c) == want
    assert bench.OPS_PHILOX == 112   # 10 rounds x (2 mul.lo + 2 mul.hi + 4 xor + 2 key adds) + 4 x 3


def test_traffic_is_keyed_to_the_kernel_sources(tmp_path, monkeypatch):
    for name in ("trace_wavefront_warp_cornell_traffic.json", "trace_wavefront_warp_sheet_traffic.json"):
        info = json.load(open(os.path.join(ROOT, "profiles", name)))
        assert info["bytes_per_launch"] > 0 and info["sources"]
        # the committed file matches the committed sources
        assert bench.kernel_traffic(name) == info["bytes_per_launch"], name
    # a changed source makes it unknown
    fake = tmp_path / "profiles"
    fake.mkdir()
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    info = {"bytes_per_launch": 123, "sources": ["k.cu"], "sources_sha256": "0" * 64}
    (fake / "t.json").write_text(json.dumps(info))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("t.json") is None
