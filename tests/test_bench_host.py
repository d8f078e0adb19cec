"""bench.py on the CPU: the oracle reference arm prints one JSON line with the
contract's keys, and the serving benchmark's arrival stream is seeded."""
import json
import os

import numpy as np
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "4x4_D2_Dc16", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["config"]["workload"] == "4x4_D2_Dc16"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_serving_stream_is_seeded_and_follows_the_mix():
    import bench
    a = bench.serving_stream(1234, 2.0, 20.0)
    b = bench.serving_stream(1234, 2.0, 20.0)
    assert a == b and len(a) > 10
    times = [x[0] for x in a]
    assert times == sorted(times) and times[-1] <= 20.0
    shapes = set(bench.SERVING_SHAPES)
    for (_, L, D, Dc, B, _) in a:
        assert (L, D, Dc) in shapes and Dc == 4 * D and B in bench.SERVING_SAMPLES
    assert bench.serving_stream(1235, 2.0, 20.0) != a
    # the mix of the serving workload: every L in {8..24} with D in {4, 6, 8},
    # Dc = 4 D, 64 to 1024 samples, weights summing to one
    assert {L for L, _, _ in bench.SERVING_SHAPES} == {8, 12, 16, 20, 24}
    assert {D for _, D, _ in bench.SERVING_SHAPES} == {4, 6, 8}
    assert min(bench.SERVING_SAMPLES) == 64 and max(bench.SERVING_SAMPLES) == 1024
    w = bench.serving_weights()
    assert abs(w.sum() - 1.0) < 1e-12 and np.all(w > 0)
    long = bench.serving_stream(7, 50.0, 200.0)
    assert len({(L, D) for (_, L, D, _, _, _) in long}) >= 9
