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


def test_study_modes_print_their_tables(monkeypatch, capsys):
    """The bond-dimension sweep, regauge-policy and degree-4 study modes, run against a stand-in
    of the library and of torch's CUDA events (no GPU): every cell of each table is present,
    with rates from the events, sweeps from the statistics, and errors against the FP64 cell."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import bench
    from paper_2409_12240_gb300 import gtqa as G

    class Ev:
        def __init__(self, **kw):
            pass

        def record(self, stream=None):
            pass

        def elapsed_time(self, other):
            return 2.0   # ms per timed layer

    class Ctx:
        def __enter__(self):
            return self

        def __exit__(self, *a):
            return False

    monkeypatch.setattr(torch.cuda, "Event", Ev)
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: type("S", (), {"cuda_stream": 0})())
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: Ctx())
    real_empty = torch.empty
    monkeypatch.setattr(torch, "empty", lambda *a, **k: real_empty(16, dtype=torch.uint8))
    sizes, sweeps, prec_of = {}, {"n": 0}, {}

    def create(n, edges, J, h, chi, colour, opt=None):
        sizes["n"] = n
        prec_of["p"] = opt
        return 1

    def stats(s):
        sweeps["n"] += 5
        return {"bp_sweeps": sweeps["n"]}

    def marginals(s):
        n = sizes["n"]
        rho = np.zeros((n, 2, 2), complex)
        rho[:, 0, 0] = 0.7 + 1e-6 * (prec_of["p"] or 0)
        rho[:, 1, 1] = 1 - rho[:, 0, 0]
        return rho, np.ones(n, np.int8)

    fakes = dict(load=lambda **k: None, gtqa_create=create, gtqa_options_init=lambda precision=0, **k: precision,
                 gtqa_anneal=lambda *a: None, gtqa_anneal_graph=lambda *a: None, gtqa_anneal_policy=lambda *a: None,
                 gtqa_trotter_layer=lambda *a: None, gtqa_residual=lambda s: 1e-3,
                 gtqa_regauge_counts=lambda s: (0, 0), gtqa_stats=stats,
                 gtqa_get_state=lambda s: (np.zeros(1), np.zeros(1), np.zeros(1)),
                 gtqa_set_state=lambda s, a, b, c: None, gtqa_destroy=lambda s: None, gtqa_marginals=marginals)
    for k, v in fakes.items():
        monkeypatch.setattr(G, k, v)
    bench.chi_sweep(None)
    t = json.loads(capsys.readouterr().out)["chi_sweep"]
    assert len(t) == 3 and all(list(c) == ["2", "4", "8", "16"] for c in t.values())
    cell = t["J~N(0,1),h~N(0,0.1)"]["4"]
    assert list(cell) == ["fp64", "mixed", "complex64"] and abs(cell["fp64"]["layers_per_s"] - 500.0) < 1e-9
    assert "max_abs" not in cell["fp64"] and abs(cell["mixed"]["max_abs"] - 1e-6) < 1e-12
    assert cell["mixed"]["bp_sweeps_per_layer"] == 5 / 40 and cell["mixed"]["sign_agreement"] == 1.0
    bench.policy_study(None)
    p = json.loads(capsys.readouterr().out)["policy_study"]
    assert list(p) == ["300", "1500", "2800"] and p["300"]["R_after_gates"] == 1e-3
    assert p["1500"]["threshold_0.01"]["against_every_layer"]["max_abs"] == 0.0
    bench.deg4_study(None)
    d = json.loads(capsys.readouterr().out)["deg4_study"]
    assert list(d) == ["fp64", "mixed", "complex64"] and abs(d["complex64"]["layers_per_s"] - 500.0) < 1e-9


def test_roofline_arithmetic():
    """The per-unit algorithmic counts of the bench against the method's cost table (edge gate
    with truncation about 2.4e5 flops, Vidal-gauge step about 5.5e4, a directed BP message
    48 chi^4 at chi = 4), and the roofline objects built from them: achieved work over the
    measured time, frac against the binding pipe's peak, and the layer's sum."""
    sys.path.insert(0, ROOT)
    import bench
    g64, g32 = bench.edge_gate_flops(4, False)
    assert g32 == 0 and abs(g64 / 2.4e5 - 1) < 0.1
    r64, r32 = bench.regauge_edge_flops(4, False)
    assert r32 == 0 and abs(r64 / 5.5e4 - 1) < 0.15
    assert bench.bp_sweep_flops(4, 1000, True) == 1000 * 3 * 48 * 4 ** 4
    m64, m32 = bench.edge_gate_flops(4, True)
    assert m64 < g64 and m32 > 0     # the mixed gate moves the SVD sweeps and Q applications to FP32
    peaks = object.__new__(bench.Peaks)
    peaks.sms, peaks.mhz, peaks.fp32_meas, peaks.fp64_meas = 152, 2070.0, 78.0, 1.25
    peaks.fp32 = 152 * 128 * 2 * 2070e6 / 1e12
    peaks.fp64 = 152 * 2 * 2 * 2070e6 / 1e12
    # (launches, total ms, units processed over those launches)
    prof = {"gates_kernel": (10, 3.0, 15000), "bp_kernel": (10, 4.0, 10000), "regauge_kernel": (10, 0.8, 15000)}
    dlt = {"svd_pairs": 0, "svd_rotations": 0, "bp_sweeps": 650, "regauge_svd_sweeps": 0}
    roofs = bench.rooflines(prof, dlt, 4, 1000, 1500, True, peaks, traffic=False)
    bp = roofs["bp_kernel"]
    assert bp["pipe"] == "fp32" and abs(bp["achieved"] - 650 * 3.6864e7 / 4e-3 / 1e12) < 1e-9
    assert abs(bp["frac"] - bp["achieved"] / peaks.fp32) < 1e-12 and bp["us_per_sweep"] == 4000 / 650
    ga = roofs["gates_kernel"]
    assert ga["pipe"] == "fp64" and abs(ga["achieved"] - 15000 * m64 / 3e-3 / 1e12) < 1e-9
    lay = bench.layer_roofline(roofs)
    t_roof = sum(r["roofline_us_per_launch"] * 10 for r in roofs.values())
    assert abs(lay["frac"] - t_roof / 7800.0) < 1e-12 and abs(lay["measured_us"] - 7800.0) < 1e-9
