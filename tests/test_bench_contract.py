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
    """The headline counts are the scope table's: 26 per tracking step (a quarter Philox block,
    a logarithm, ~10 FP32), 78 more per real event, 45 per connection, 26 per ratio-tracking step;
    cell walks (an optimisation) count nothing."""
    c = {"steps": 10, "events": 3, "connections": 2, "connect_steps": 8, "cell_walks": 5}
    assert bench.algorithmic_ops(c) == 10 * 26 + 3 * 78 + 2 * 45 + 8 * 26
    assert bench.mufu_ops(c) == 10 * 1 + 3 * 3 + 2 * 2 + 8 * 1
    assert bench.OPS_PHILOX == 112   # 10 rounds x (2 mul.lo + 2 mul.hi + 4 xor + 2 key adds) + 4 x 3
    assert bench.rng_contract_ops(c) == 10 * 167 + 3 * 142 + 2 * 45 + 8 * 64
    alu, mufu, rng = bench.rooflines(c, 1e-6, 152, 2070.0)
    assert abs(alu["frac"] - bench.algorithmic_ops(c) / 1e-6 / (152 * 128 * 2070e6)) < 1e-12
    assert abs(mufu["frac"] - bench.mufu_ops(c) / 1e-6 / (152 * 16 * 2070e6)) < 1e-12
    assert rng["frac"] > alu["frac"]


def test_traffic_is_keyed_to_the_kernel_sources(tmp_path, monkeypatch):
    for name in ("trace_wavefront_warp_cornell_traffic.json", "trace_wavefront_warp_sheet_traffic.json"):
        info = json.load(open(os.path.join(ROOT, "profiles", name)))
        assert info["bytes_per_launch"] > 0 and info["sources"]
        # the committed figure while the sources match, else unknown
        assert bench.kernel_traffic(name) in (info["bytes_per_launch"], None), name
    fake = tmp_path / "profiles"
    fake.mkdir()
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    import hashlib
    good = hashlib.sha256(b"kernel v1").hexdigest()
    (fake / "t.json").write_text(json.dumps({"bytes_per_launch": 123, "sources": ["k.cu"],
                                             "sources_sha256": good}))
    (fake / "p.json").write_text(json.dumps({"metrics": {"x": 1}, "sources": ["k.cu"],
                                             "sources_sha256": good}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("t.json") == 123
    assert bench.kernel_profile("p.json") == {"x": 1}
    # a changed source makes both unknown
    src.write_text("kernel v2")
    assert bench.kernel_traffic("t.json") is None
    assert bench.kernel_profile("p.json") is None


def test_launch_count_includes_the_film_folds():
    """Every render with a film launches the trace kernel and the fold of its fixed-point film sums;
    the batch and the adjoint have no film."""
    assert bench.FILM_RENDER_LAUNCHES == 2
    none = bench.count_launches(20, 10, None, None, None, 3, None, None, None, 3)
    assert none == 2 * (2 * 20 + 10)
    n = bench.count_launches(20, 10, {"steps": 3, "plain_launches": 256}, {"launches_per_step": 5},
                             {"launches_per_step": 2}, 3, {"launches_per_step": 2, "steps": 2},
                             {"launches_per_step": 2, "steps": 2}, {"launches": 12}, 3)
    assert n == none + (3 + 256) + 5 * 3 + 2 * 2 * 3 + 2 * (2 + 1) + 2 * (2 + 1) + 12
