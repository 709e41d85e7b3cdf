"""Host-side checks of the benchmark contract and of the loud failure without
the CUDA library (no GPU needed)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "uniform_1000x800x600_100k_r16", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["config"]["workload"] == "uniform_1000x800x600_100k_r16"


def test_warmup_below_three_is_refused():
    import bench
    with pytest.raises(SystemExit):
        bench.parse_args(["--warmup", "2"])


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2309_09131_gb300 import _native
    monkeypatch.setattr(_native, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_native, "_lib", None)
    with pytest.raises(ImportError):
        _native.lib()


def test_profiled_traffic_is_plausible_for_the_current_kernel():
    # the bench's roofline "traffic" comes from the committed ncu summary only
    # when it was captured on this exact kernel source; then it must sit near
    # the algorithmic bytes of a 77M-nonzero pass: at most 2x, and at least 0.9x
    # (a pass ends with part of its remap writes still in L2; they reach DRAM
    # during the next launch, so one launch's counters can read a little low)
    import bench
    # the bench tensor's default shard size: 77M nonzeros over 3 x 152 bins
    t = bench.traffic_from_profiles(bench.kernel_source_sha(), 8192)
    if t is None:
        pytest.skip("the committed ncu summary predates the current kernel source")
    per_mode, _ = bench.step_bytes((12000, 9000, 29000), 77_000_000, 32, 4, 16)
    alg = sum(per_mode) / 3
    assert 0.9 * alg <= t <= 2 * alg, (t, alg)
