"""bench.py's reference arm (the CPU oracle) prints the contract's JSON line (CPU only)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "tiny", "--steps", "2", "--warmup", "3"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["unit"] == "GB/s" and d["value"] > 0 and d["steps"] == 2 and d["warmup"] >= 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_cpu_baseline_object_of_the_gpu_line():
    """The cpu_baseline object of the GPU arm's line: the oracle on all host
    threads and its one-thread rate, and beside it the paper's closed-form
    rearrangement (Sec. 4) on all cores and on one."""
    sys.path.insert(0, ROOT)
    import bench
    import lfgen
    specs = lfgen.config_specs("tiny")
    Hs = [lfgen.generate(s).numpy() for s in specs]
    d = bench._cpu_oracle_rate(specs, Hs, None, budget_s=0.5, max_passes=4)
    assert d["kind"] == "oracle" and d["unit"] == "GB/s" and d["cores"] >= 1
    for key in ("value", "single_thread_GBps"):
        assert d[key] > 0, key
    assert "oracle.transpose" in d["sample"]
    cf = d["closed_form"]
    assert cf["unit"] == "GB/s" and cf["cores"] >= 1
    assert cf["value"] > 0 and cf["single_thread_GBps"] > 0


def test_summary_is_last_and_compact():
    """The forms side by side come last on the line, so that the tail of the
    output shows them."""
    sys.path.insert(0, ROOT)
    import bench
    line = {"value": 5000.0, "plain": {"value": 4000.0}, "roofline": {"frac": 0.7},
            "extra": {"ragged": {"batched_GBps": 4500.0, "plain_GBps": 2800.0},
                      "highres_fp16": {"batched_GBps": 4300.0, "plain_GBps": 3300.0},
                      "mid": {"batched_GBps": 4100.0, "plain_GBps": 3900.0},
                      "paper_window": {"even_K": {"batched_GBps": 4000.0, "plain_GBps": 3000.0}}},
            "cpu_baseline": {"value": 20.0, "cores": 16,
                             "closed_form": {"value": 30.0, "single_thread_GBps": 3.0}}}
    sm = bench._summary(line)
    assert sm["ragged"] == {"batched": 4500.0, "plain": 2800.0}
    assert sm["mid"]["plain"] == 3900.0 and sm["even_K"]["batched"] == 4000.0
    assert sm["cpu_GBps"]["closed_form"] == 30.0 and sm["cpu_GBps"]["cores"] == 16
    assert len(json.dumps(sm)) < 700
