"""The reference arm of bench.py (the CPU oracle, timed on a bounded sample of the headline
workload) prints one JSON line with the keys the measurement contract names."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "layers/s"
    assert line["higher_is_better"] is True and line["n_gpus"] == 1 and line["steps"] == 1
    assert line["warmup"] == 3 and "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_timed_layers_spread_over_the_anneal():
    """A short run samples the whole anneal (first and last layer included); the default run
    times every layer after the warm-up."""
    sys.path.insert(0, ROOT)
    import bench
    L = bench.sample_layers(5, 20, 3200)
    assert len(L) == 20 and L[0] == 6 and L[-1] == 3200 and L == sorted(set(L))
    assert max(b - a for a, b in zip(L, L[1:])) - min(b - a for a, b in zip(L, L[1:])) <= 1
    assert bench.sample_layers(3, 3197, 3200) == list(range(4, 3201))
    assert bench.sample_layers(3, 1, 3200) == [3200]
    assert bench.spread(list(range(100)), 5) == [0, 25, 50, 74, 99]
    assert bench.spread([1, 2, 3], 5) == [1, 2, 3]
