"""bench.py's reference arm (the FP64 oracle timed on the host cores) keeps the
benchmark's JSON-line contract; it needs no GPU, so it runs here on a small set."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                        "--workload", "uniform-32k"], cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env={**os.environ, "CUDA_VISIBLE_DEVICES": ""})
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["unit"] == "forces/s" and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("uniform-32k")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_cpu_baseline_leg_returns_the_accuracy_reference():
    """The CPU-baseline leg times the oracle's direct sum on the accuracy sinks and
    on random ones, and hands back the accuracy sinks' forces: equal to a direct
    call on them, and counted in the baseline's sample."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_2006_14952_gb300 import workloads as W

    cfg = W.CONFIGS["uniform-32k"]
    pos, mass = W.make(cfg)
    sinks = W.subsample(cfg.n, 300, 2024)
    rec, ref = bench.cpu_oracle_sample(pos, mass, cfg, 0.2, fixed_sinks=sinks)
    np.testing.assert_array_equal(ref, oracle.direct_sr(pos, mass, cfg.box, cfg.rs, cfg.rc, sinks=sinks))
    assert rec["kind"] == "oracle" and rec["value"] > 0 and "300 fixed (accuracy)" in rec["sample"]
    rec2, ref2 = bench.cpu_oracle_sample(pos, mass, cfg, 0.2)
    assert ref2 is None and "0 fixed" in rec2["sample"]
