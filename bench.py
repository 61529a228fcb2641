#!/usr/bin/env python3
"""Throughput of the GTQA hot path: Trotter layers per second on one GB300.

Workload (the single-instance annealing run): seeded random 3-regular graph with
n = 1000 vertices (m = 1500 edges, 3-colour matching schedule from a Kempe-chain edge colouring),
J_ab ~ N(0, 1), h_a ~ N(0, 0.1), bond dimension chi = 4, linear schedule over
K = 3200 Trotter layers with dt = 0.2, BP tolerance 1e-8 (at most 100 sweeps).
One step = one full annealing layer: every edge gate with truncation, the mixing
layer, flooding BP to tolerance from the warm start, and Vidal-gauge finding.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
    python bench.py --impl reference ...     # the CPU oracle on the same workload

Prints one JSON line (rank 0).  Under torchrun every rank runs its own replica of
the workload (no collective on the data path) and the slowest rank's time counts.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np
from typing import Tuple

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Trotter layers/sec at n=1000, chi=4 (mixed vs FP64 GPU) at stated marginal error"
WL = dict(n=1000, seed=0, chi=4, K=3200, dt=0.2, tol=1e-8, max_iter=100)
WORKLOAD_NAME = ("random 3-regular n=1000 (m=1500, 3-colour schedule), J~N(0,1), h~N(0,0.1), "
                 "chi=4, K=3200 layers, dt=0.2, BP tol 1e-8, max 100 sweeps")
L2_FLUSH_BYTES = 256 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gtqa", choices=["gtqa", "reference"])
    p.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64-path comparison run")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--ncu-scale", type=int, default=None, metavar="N",
                   help="short run of the chi = 8 scale configuration's shape at n = N for ncu: five "
                        "layers, then one gates, one BP (10 sweeps) and one regauge launch")
    p.add_argument("--ncu-case", type=int, default=None, metavar="K0",
                   help="profiling case: anneal layers 1..K0, then one gates launch, one BP launch of 1 sweep "
                        "and, from the same state, one of 21 sweeps (warm start, no regauge); no timing")
    p.add_argument("--budget", type=float, default=15.0, help=argparse.SUPPRESS)
    a = p.parse_args()
    if a.steps is None:
        a.steps = WL["K"] - a.warmup
    a.warmup = max(0, a.warmup)
    if a.warmup + a.steps > WL["K"]:
        a.steps = max(1, WL["K"] - a.warmup)
    return a


def instance():
    from instances import make_instance
    return make_instance(WL["n"], WL["seed"])


# ---------------------------------------------------------------------------
# CPU oracle, timed on a bounded sample of the workload
# ---------------------------------------------------------------------------
def oracle_sampled_rate(W: int, K: int, budget_s: float) -> dict:
    """Layers/s of the CPU oracle on this workload.

    W full oracle layers (k = 1..W) are run first.  Each of the K steps then times a
    fraction f of one layer's per-unit work with the oracle's own functions: the gates
    of f*m edges (in schedule order), the mixing gate on the matching share of
    vertices, the symmetric split of the touched vertices, s BP message updates of
    the 2 f m directed messages of those edges (s = sweeps the last full layer used),
    and the per-edge Vidal-gauge step of those edges.  value = sum of fractions /
    sum of times.  f is chosen so the K steps take about budget_s seconds.
    """
    from oracle import gtqa_oracle as O
    inst = instance()
    n, m = inst.n, inst.m
    st = O.plus_state(n, inst.edges)
    deg = [len(x) for x in st.inc]
    t_layer, s_ref = None, 1
    for k in range(1, max(W, 1) + 1):
        tZ, tX = O.schedule(k, WL["K"], WL["dt"])
        t0 = time.perf_counter()
        st, info = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, WL["chi"], WL["tol"], WL["max_iter"])
        t_layer = time.perf_counter() - t0
        s_ref = max(1, int(info["bp_iters"]))
    f = min(1.0, budget_s / (K * t_layer))
    q = max(1, int(round(f * m)))
    order = sorted(range(m), key=lambda e: (int(inst.colour[e]), e))
    tot_t, tot_units = 0.0, 0.0
    for j in range(K):
        k = min(WL["K"], max(W, 1) + 1 + j)
        tZ, tX = O.schedule(k, WL["K"], WL["dt"])
        sel = [order[(j * q + i) % m] for i in range(q)]
        verts = sorted({int(x) for e in sel for x in inst.edges[e]})
        t0 = time.perf_counter()
        for e in sel:
            a, b = int(inst.edges[e][0]), int(inst.edges[e][1])
            Wg = O.ising_gate(float(inst.J[e]), float(inst.h[a]), float(inst.h[b]), deg[a], deg[b], tZ)
            O.simple_update(st, e, Wg, WL["chi"])
        Wx = O.mixing_gate(tX)
        for a in verts[: max(1, int(round(q * n / m)))]:
            O.apply_single_qubit_gate(st, a, Wx)
        T = {a: O.symmetric_gauge_vertex(st, a) for a in verts}
        msgs = {}
        for a in verts:
            for e in st.inc[a]:
                lam = st.lam[e]
                mm = np.diag(lam / lam.sum()).astype(np.complex128)
                msgs[(e, 0)] = mm
                msgs[(e, 1)] = mm
        new = {}
        for _ in range(s_ref):
            for e in sel:
                for a in (int(inst.edges[e][0]), int(inst.edges[e][1])):
                    key = O.directed(st, a, e)
                    mm = O.message_update(st, T, msgs, a, e)
                    mm = mm / np.trace(mm)
                    O.trace_norm(mm - msgs[key])
                    new[key] = mm
        view = O.VidalState(st.n, st.edges, st.inc, dict(T), {e: st.lam[e] for a in verts for e in st.inc[a]})
        for e in sel:
            O.vidal_gauge_edge(view, e, new)
        tot_t += time.perf_counter() - t0
        tot_units += q / m
    return {"value": tot_units / tot_t, "unit": "layers/s", "cores": 1, "kind": "oracle",
            "sample": (f"{max(W, 1)} full oracle layers from |+>, then {K} steps each timing {q} of {m} edges' "
                       f"gate, {s_ref} BP update(s) of their {2 * q} directed messages, symmetric split, mixing "
                       f"and regauge (fraction {q / m:.4f} of a layer per step), scaled to whole layers"),
            "seconds": tot_t}


def cpu_baseline_subprocess(W: int, budget: float) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    env.pop("WORLD_SIZE", None)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-sample", "--warmup", str(W),
           "--steps", "20", "--budget", str(budget)]
    r = subprocess.run(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, timeout=900)
    if r.returncode != 0:
        return {"value": None, "error": r.stderr.decode(errors="replace")[-400:]}
    return json.loads(r.stdout.decode().strip().splitlines()[-1])


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS),
                                       "--format=csv,noheader,nounits", "-lms", "200", "-i", str(self.index)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.decode(errors="replace").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic work per unit (flop counts of the variant that runs)
# ---------------------------------------------------------------------------
def storage_chi(chi: int) -> int:
    return 2 if chi <= 2 else (4 if chi <= 4 else 8)


def gate_flops(chi: int, edges: int, pairs: int, rotations: int, mixed: bool = False):
    """FP64 flops of the simple-update phase (real adds/muls, fma = 2).

    Per edge at storage bond dimension C (rows R = C^2 per QR block, N = 2C):
      X = Gamma * lambda products  8C^3 + 2C^2
      Householder QR of 4 blocks   4 sum_k [3(R-k) + 16 (R-k)(C-1-k)]
      core M (triangular R's)      sum_{r,r'} 10 (C - max(r, r')) + 26 per entry, 4 blocks
      singular values              3 N^2
      Q U / lambda (4 blocks)      4 C sum_k 16 (R-k) + 8 C R
    plus per Jacobi pair examined 14 N (alpha, beta, gamma) and per rotation 40 N + 15.
    Returns (FP64 flops, FP32 flops).  In the mixed mode the counted Jacobi sweeps are the
    FP64 polish after the FP32 preconditioning sweeps (which are not counted), the
    Newton-Schulz step (V^H V, V(3I - G)/2) and W = M V add 3 x 8 N^3 FP64 flops per
    edge, and the last line (Q U / lambda) runs in FP32.
    """
    C = storage_chi(chi)
    R, N = C * C, 2 * C
    x = 8 * C ** 3 + 2 * C * C
    qr = 4 * sum(3 * (R - k) + 16 * (R - k) * (C - 1 - k) for k in range(C))
    core = 4 * sum(10 * (C - max(r, rp)) + 26 for r in range(C) for rp in range(C))
    sv = 3 * N * N
    back = 4 * C * sum(16 * (R - k) for k in range(C)) + 8 * C * R
    jac = pairs * 14 * N + rotations * (40 * N + 15)
    if not mixed:
        return float(edges * (x + qr + core + sv + back) + jac), 0.0
    ns = 3 * 8 * N ** 3
    return float(edges * (x + qr + core + sv + ns) + jac), float(edges * back)


def bp_sweep_flops(chi: int, vertices: int, mixed: bool) -> float:
    """Algorithmic flops of one flooding sweep (Eq. local_consistency) over `vertices` vertices
    of degree 3: per directed message 3 contractions of 2 chi^4 complex MACs = 48 chi^4 real
    flops (the per-message figure of the method; FP32 in the mixed mode).  The mixed kernel
    executes 4 contractions per message (64 chi^4, the delta-form update) and replaces the
    per-message FP64 trace-norm eigen-decomposition by a bound; neither difference is counted."""
    return float(vertices * 3 * 48 * chi ** 4)


def edge_gate_flops(chi: int) -> Tuple[float, float]:
    """Algorithmic flops of one edge gate with truncation (a2-a3), in complex MACs of 8 flops:
    two Householder QRs of the (2 chi^2) x (2 chi) side matrices (2 m n^2 - 2/3 n^3 each), the
    core M (2 (2 chi)^3), a one-sided Jacobi SVD of order n = 2 chi with V (11 n per pair, 7.5
    sweeps of n (n - 1) / 2 pairs), the two Q applications (2 chi (m n - n^2 / 2) each), plus
    about 50 chi^3 flops of gate and lambda scaling.  Returns (total, FP64 part = 95 %)."""
    m, n = 2 * chi * chi, 2 * chi
    cmac = 2 * (2 * m * n * n - 2 * n ** 3 / 3) + 2 * n ** 3 + 11 * n * (n * (n - 1) / 2) * 7.5 \
        + 2 * 2 * chi * (m * n - n * n / 2)
    tot = 8 * cmac + 50 * chi ** 3
    return float(tot), float(0.95 * tot)


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_n1000_chi4.json")
TRAFFIC_SOURCES = [os.path.join(ROOT, "paper_2409_12240_gb300", "csrc", f) for f in ("gtqa_anneal.cuh", "gtqa_common.cuh")]


def kernel_traffic(kernel: str, mixed: bool, chi: int, sweeps_per_launch: float = 0.0):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the committed
    ncu capture of `bench.py --ncu-case`; BP launches are scaled to this run's sweeps per launch
    from the captured 1-sweep and 21-sweep launches.  None if there is no capture for this mode
    or the kernel sources changed since it was taken."""
    import hashlib
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    h = hashlib.sha256()
    for p in TRAFFIC_SOURCES:
        with open(p, "rb") as f:
            h.update(f.read())
    r = rec.get("mixed" if mixed else "fp64")
    if not r or r.get("sources_sha256") != h.hexdigest() or r.get("chi") != chi or kernel not in r:
        return None
    k = r[kernel]
    if kernel == "bp_kernel":
        return k["fixed_bytes"] + k["bytes_per_sweep"] * sweeps_per_launch
    return k["bytes_per_launch"]


def per_layer_error(G, make, inst, k_last: int, samples: int = 6) -> dict:
    """Marginal error introduced by one mixed-precision layer: at sampled layers k the
    FP64 state after layer k-1 is loaded into a mixed and an FP64 state, layer k runs in
    both, and max |rho_mixed - rho_fp64| over vertices is recorded."""
    Ks, dt, tol, mi = WL["K"], WL["dt"], WL["tol"], WL["max_iter"]
    ks = sorted({max(2, int(round(k_last * (i + 1) / samples))) for i in range(samples)})
    ref = make(G.GTQA_FP64)
    out, done = {}, 0
    try:
        for k in ks:
            G.gtqa_anneal(ref, done + 1, k - 1, Ks, dt, tol, mi)
            done = k - 1
            Gm, L, Mg = G.gtqa_get_state(ref)
            errs = []
            rhos = []
            for p in (G.GTQA_MIXED, G.GTQA_FP64):
                s = make(p)
                G.gtqa_set_state(s, Gm, L, Mg)
                G.gtqa_anneal(s, k, k, Ks, dt, tol, mi)
                rhos.append(G.gtqa_marginals(s))
                G.gtqa_destroy(s)
            (rm, sm_), (rf, sf) = rhos
            clear = np.abs(rf[:, 0, 0].real - 0.5) > 1e-3
            out[str(k)] = {"max_abs": float(np.abs(rm - rf).max()),
                           "sign_agreement": float(np.mean(sm_[clear] == sf[clear]))}
    finally:
        G.gtqa_destroy(ref)
    return {"max_abs": max(v["max_abs"] for v in out.values()),
            "min_sign_agreement": min(v["sign_agreement"] for v in out.values()), "samples": out,
            "note": "one layer in each mode from the same FP64 state at layer k-1"}


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------
def replica_throughput(t_ms: float, K: int, world: int, dist=None, device: str = "cpu"):
    """Whole-job throughput of `world` independent replicas that each ran K layers: the slowest
    rank's time (max over ranks), and value = world * K layers / that time."""
    if dist is not None and world > 1:
        import torch
        tt = torch.tensor([t_ms], device=device, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
    return t_ms, world * K / (t_ms / 1e3)


def run_gtqa(a):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2409_12240_gb300 import gtqa as G
    G.load(build_if_missing=True)
    mixed = a.precision == "mixed"
    prec = G.GTQA_MIXED if mixed else G.GTQA_FP64
    inst = instance()
    W, K = a.warmup, a.steps
    Ks, dt, tol, mi, chi = WL["K"], WL["dt"], WL["tol"], WL["max_iter"], WL["chi"]

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu = cpu_baseline_subprocess(W, a.budget)

    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def make(p):
        return G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour,
                             G.gtqa_options_init(precision=p, cuda_stream=stream.cuda_stream))

    def timed_window(p, clocks=None, profile=False):
        """Warm-up layers 1..W, then layers W+1..W+K, one gtqa_anneal call per layer with an
        L2 flush between layers (outside the events).  With `profile`, the library also
        records CUDA events around each of its launches on the same stream (the per-kernel
        durations of the roofline).  Returns (ms, stats delta, final rho, sign, clocks, prof)."""
        s = make(p)
        if W:
            G.gtqa_anneal(s, 1, W, Ks, dt, tol, mi)
        if profile:
            G.gtqa_profile(s, True)
        st0 = G.gtqa_stats(s)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        with torch.cuda.stream(stream):
            for j in range(K):
                flush.fill_(j & 0xFF)
                ev[j][0].record(stream)
                G.gtqa_anneal(s, W + 1 + j, W + 1 + j, Ks, dt, tol, mi)
                ev[j][1].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ck = clocks.stop() if clocks else None
        t_ms = float(sum(e0.elapsed_time(e1) for e0, e1 in ev))
        prof = G.gtqa_profile_read(s) if profile else None
        st1 = G.gtqa_stats(s)
        rho, sign = G.gtqa_marginals(s)
        G.gtqa_destroy(s)
        delta = {k: st1[k] - st0[k] for k in ("launches", "bp_sweeps", "bp_calls", "bp_not_converged_calls",
                                               "svd_pairs", "svd_rotations")}
        return t_ms, delta, rho, sign, ck, prof

    clocks = Clocks(local)
    t_ms, dlt, rho_main, sign_main, ck, prof = timed_window(prec, clocks, profile=True)
    t_ms, value = replica_throughput(t_ms, K, world, dist, "cuda")

    # the FP64 path on the same layers, and the marginal error of the mixed path against it
    fp64 = None
    if mixed and not a.no_fp64:
        t64, d64, rho64, sign64, _, _ = timed_window(G.GTQA_FP64)
        err = np.abs(rho_main - rho64)
        clear = np.abs(rho64[:, 0, 0].real - 0.5) > 1e-3
        fp64 = {"value": world * K / (t64 / 1e3), "unit": "layers/s", "ms_per_step": t64 / K,
                "bp_sweeps_per_layer": d64["bp_sweeps"] / K,
                "speedup_mixed_over_fp64": t64 / t_ms,
                "marginal_error_per_layer": per_layer_error(G, make, inst, W + K),
                "trajectory_divergence_at_last_layer": {
                    "max_abs": float(err.max()), "mean_abs": float(err.mean()),
                    "sign_agreement": float(np.mean(sign_main[clear] == sign64[clear])), "at_layer": W + K,
                    "note": "whole trajectories; BP stops at max_iter in part of the anneal, after which both "
                            "runs follow the chaotic BP map and decorrelate"}}

    # ---- roofline of the kernel with the largest share of the timed window ----
    total_prof = sum(v[1] for v in prof.values())
    dom = max(prof, key=lambda k: prof[k][1])
    # ALU peaks derived from unit counts and the maximum SM clock: 128 FP32 lanes and 2 FP64
    # FMA units per SM, 2 flops per FMA; the FMA microbenchmark is reported beside them
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = (ck or {}).get("sm_max_mhz") or 2070.0
    fp32_peak = sms * 128 * 2 * mhz * 1e6 / 1e12
    fp64_peak = sms * 2 * 2 * mhz * 1e6 / 1e12
    fp64_meas = G.gtqa_alu_peak(True)
    fp32_meas = G.gtqa_alu_peak(False)
    peak_note = f"{sms} SMs x {{lanes}} x 2 flop x {mhz:.0f} MHz (derived); FMA microbenchmark {{meas:.3f}} TFLOP/s"
    def roofline_of(kname):
        nl, ms, units = prof[kname]
        if not nl:
            return None
        if kname == "gates_kernel":
            _, f64e = edge_gate_flops(chi)
            f64 = f64e * units
            ach = f64 / (ms * 1e-3) / 1e12
            return {"kernel": kname, "bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": ach / fp64_peak, "traffic": kernel_traffic(kname, mixed, chi),
                    "peak_source": peak_note.format(lanes="2 FP64 FMA units", meas=fp64_meas),
                    "algorithmic_flops_per_launch": f64 / nl, "avg_launch_us": ms / nl * 1e3,
                    "unit_count": "edges per launch x the FP64 part (95 %) of the edge gate's algorithmic flops",
                    "executed_fp64_flops_per_launch": gate_flops(chi, units, int(dlt["svd_pairs"]),
                                                                 int(dlt["svd_rotations"]), mixed)[0] / nl,
                    "note": "the mixed path runs the SVD's preconditioning sweeps in FP32, so it executes fewer "
                            "FP64 flops than it is credited with; the frac is against the FP64 peak"}
        if kname == "bp_kernel":
            sweeps = int(dlt["bp_sweeps"])
            fl = bp_sweep_flops(chi, inst.n, mixed) * sweeps
            peak = fp32_peak if mixed else fp64_peak
            ach = fl / (ms * 1e-3) / 1e12
            return {"kernel": kname, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": kernel_traffic(kname, mixed, chi, sweeps / nl),
                    "peak_source": peak_note.format(lanes="128 FP32 lanes" if mixed else "2 FP64 FMA units",
                                                    meas=fp32_meas if mixed else fp64_meas),
                    "algorithmic_flops_per_launch": fl / nl, "avg_launch_us": ms / nl * 1e3,
                    "sweeps_per_launch": sweeps / nl, "us_per_sweep": ms * 1e3 / max(sweeps, 1),
                    "unit_count": "sweeps x 3n directed messages x 48 chi^4 flops",
                    "note": "flops of the BP sweeps only (the warm-start phase of each launch is not counted); "
                            "the working set is L2-resident and each sweep is bounded by a grid barrier"}
        return None

    roof = roofline_of(dom)
    roof_other = {k: roofline_of(k) for k in ("gates_kernel", "bp_kernel") if k != dom and k in prof}
    kernel_share = {k: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / total_prof, 4) if total_prof else 0}
                    for k, v in prof.items() if v[0]}

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if not a.no_e2e:
        rho_h = torch.empty((inst.n, 2, 2), dtype=torch.complex128, pin_memory=True).numpy()
        sign_h = torch.empty(inst.n, dtype=torch.int8, pin_memory=True).numpy()
        h2d = inst.edges.nbytes + inst.J.nbytes + inst.h.nbytes + inst.colour.nbytes
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s3 = make(prec)
        for j in range(K):
            G.gtqa_anneal(s3, j + 1, j + 1, Ks, dt, tol, mi)
            G.gtqa_marginals(s3, rho_h, sign_h)
        G.gtqa_destroy(s3)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        e2e = {"value": world * K / t_e2e, "unit": "layers/s", "h2d_bytes_per_step": h2d / K,
               "d2h_bytes_per_step": rho_h.nbytes + sign_h.nbytes,
               "note": "create from host arrays, layers 1..K each followed by marginals into pinned host buffers, destroy"}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    out = {
        "metric": METRIC, "value": value, "unit": "layers/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": t_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64/f64" if mixed else "c128/f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "precision": a.precision, "layers_timed": [W + 1, W + K],
                   "l2": "flushed between timed layers (256 MiB write, outside the timed events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "bp_sweeps_per_layer": dlt["bp_sweeps"] / K,
        "bp_layers_at_max_iter": dlt["bp_not_converged_calls"] / K,
        "fp64_path": fp64,
        "roofline": roof, "roofline_other_kernels": roof_other, "kernel_share": kernel_share, "alu_peaks_tflops": {"fp32": fp32_peak, "fp64": fp64_peak, "fp32_measured": fp32_meas,
                             "fp64_measured": fp64_meas},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(dlt["launches"]), "clocks": ck,
        "final_marginals": {"mean_abs_z": float(np.mean(np.abs(rho_main[:, 0, 0].real - rho_main[:, 1, 1].real)))},
    }
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    W, K = a.warmup, a.steps
    r = oracle_sampled_rate(W, K, budget_s=120.0)
    out = {"impl": "reference", "metric": METRIC, "value": r["value"], "unit": "layers/s", "n_gpus": world,
           "steps": K, "warmup": W, "ms_per_step": 1e3 / r["value"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "c128/f64", "data": "synthetic",
           "config": {"workload": WORKLOAD_NAME, "precision": "fp64 (CPU oracle)", "layers_timed": [W + 1, W + K]},
           "cpu_baseline": {"value": r["value"], "unit": "layers/s", "cores": 1, "kind": "oracle", "sample": r["sample"]},
           "e2e": {"value": r["value"], "unit": "layers/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def ncu_case(a):
    """A short run for ncu captures: the launches of interest come after 3 K0 warm-up launches
    (gates, BP, regauge per layer); the gates launch is the (K0+1)-th gates_kernel, the two BP
    launches the (K0+1)-th and (K0+2)-th bp_kernel."""
    from paper_2409_12240_gb300 import gtqa as G
    G.load(build_if_missing=True)
    inst = instance()
    prec = G.GTQA_MIXED if a.precision == "mixed" else G.GTQA_FP64
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, WL["chi"], inst.colour, G.gtqa_options_init(precision=prec))
    try:
        K0 = a.ncu_case
        if K0 > 0:
            G.gtqa_anneal(s, 1, K0, WL["K"], WL["dt"], WL["tol"], WL["max_iter"])
        G.gtqa_trotter_layer(s, (K0 + 1) / WL["K"], WL["dt"])
        Gm, L, M = G.gtqa_get_state(s)
        G.gtqa_bp_sweep(s, 0.0, 1, G.GTQA_BP_WARM_START)
        G.gtqa_set_state(s, Gm, L, M)
        G.gtqa_bp_sweep(s, 0.0, 21, G.GTQA_BP_WARM_START)
    finally:
        G.gtqa_destroy(s)
    print(json.dumps({"ncu_case": a.ncu_case, "precision": a.precision}))


def ncu_scale(a):
    """The shape of the n = 100000, chi = 8 configuration (random 3-regular, seed 2, J ~ N(0,1),
    h ~ N(0, 0.1), mixed, K = 500, dt = 0.05) at n = a.ncu_scale: layers 1..5 (15 launches), then
    the gates of layer 6, a 10-sweep BP launch from the warm start and a regauge launch."""
    from paper_2409_12240_gb300 import gtqa as G
    from instances import make_instance
    G.load(build_if_missing=True)
    inst = make_instance(a.ncu_scale, 2)
    K, dt, tol, mi = 500, 0.05, 1e-8, 100
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 8, inst.colour, G.gtqa_options_init(precision=G.GTQA_MIXED))
    try:
        G.gtqa_anneal(s, 1, 5, K, dt, tol, mi)
        G.gtqa_trotter_layer(s, 6 / K, dt)
        G.gtqa_bp_sweep(s, 0.0, 10, G.GTQA_BP_WARM_START)
        G.gtqa_regauge(s)
        G.gtqa_marginals(s)
    finally:
        G.gtqa_destroy(s)
    print(json.dumps({"ncu_scale": a.ncu_scale, "chi": 8, "precision": "mixed"}))


def main():
    a = parse()
    if a.ncu_case is not None:
        ncu_case(a)
        return
    if a.ncu_scale is not None:
        ncu_scale(a)
        return
    if a.oracle_sample:
        r = oracle_sampled_rate(a.warmup, a.steps, a.budget)
        print(json.dumps(r))
        return
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gtqa(a)


if __name__ == "__main__":
    main()
