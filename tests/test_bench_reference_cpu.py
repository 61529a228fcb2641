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


def _ncu_csv(path, launches):
    rows = ['==PROF== Connected to process 1 (python3)',
            '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
            '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"']
    for i, (k, r, w) in enumerate(launches):
        for mn, v in (("dram__bytes_read.sum", r), ("dram__bytes_write.sum", w)):
            rows.append(f'"{i}","1","python3","h","void {k}<4, ModeMixed, 1>(Ctx)","1","7","(256, 1, 1)",'
                        f'"(152, 1, 1)","0","10.3","Command line profiler metrics","{mn}","byte","{v:,}"')
    with open(path, "w") as f:
        f.write("\n".join(rows) + "\n")


def test_traffic_record_from_an_ncu_csv(tmp_path, monkeypatch):
    """The traffic record written from ncu's CSV of the four captured launches: per-launch DRAM
    bytes, BP split into a fixed part and a part per sweep, tagged with the hash of the current
    phase-kernel sources, which the bench's lookup then accepts; a record with another hash, or
    a capture of other launches, gives nothing."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "rec.json"))
    csv = tmp_path / "t.csv"
    _ncu_csv(csv, [("gates_kernel", 1000, 24), ("bp_kernel", 2000, 0), ("bp_kernel", 2400, 200),
                   ("regauge_kernel", 3000, 5)])
    rec = bench.traffic_record(str(csv))["mixed"]
    assert rec["gates_kernel"]["bytes_per_launch"] == 1024 and rec["regauge_kernel"]["bytes_per_launch"] == 3005
    assert rec["bp_kernel"]["bytes_per_sweep"] == 30 and rec["bp_kernel"]["fixed_bytes"] == 1970
    assert bench.kernel_traffic("bp_kernel", True, 4, 10) == 1970 + 300
    assert bench.kernel_traffic("gates_kernel", True, 4) == 1024
    assert bench.kernel_traffic("gates_kernel", False, 4) is None   # no FP64 capture
    assert bench.kernel_traffic("gates_kernel", True, 8) is None
    data = json.loads((tmp_path / "rec.json").read_text())
    data["mixed"]["sources_sha256"] = "0" * 64
    (tmp_path / "rec.json").write_text(json.dumps(data))
    assert bench.kernel_traffic("gates_kernel", True, 4) is None
    _ncu_csv(csv, [("gates_kernel", 1, 0), ("bp_kernel", 1, 0), ("regauge_kernel", 1, 0)])
    try:
        bench.traffic_record(str(csv))
    except ValueError:
        pass
    else:
        raise AssertionError("a capture of three launches was accepted")
