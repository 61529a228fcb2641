#!/usr/bin/env python3
"""Throughput of the GTQA hot path: Trotter layers per second on one GB300.

Workload (the single-instance annealing run): seeded random 3-regular graph with
n = 1000 vertices (m = 1500 edges, 3-colour matching schedule from a Kempe-chain edge colouring),
J_ab ~ N(0, 1), h_a ~ N(0, 0.1), bond dimension chi = 4, linear schedule over
K = 3200 Trotter layers with dt = 0.2, BP tolerance 1e-8 (at most 100 sweeps).
One step = one full annealing layer: every edge gate with truncation, the mixing
layer, flooding BP to tolerance from the warm start, and Vidal-gauge finding, replayed
from the library's one-layer CUDA graph.

Every run walks the whole anneal (layers 1..K).  With --steps S < K - W the S timed layers
are spread evenly over W+1..K (the layers between them run untimed), so a short run samples
the early, middle and late anneal alike; with S = K - W (the default) every layer after the
warm-up is timed.

    python bench.py [--gpus N] [--steps S] [--warmup W] [--precision fp64|mixed]
    python bench.py --impl reference ...     # the CPU oracle on the same workload

Prints one JSON line (rank 0).  Under torchrun every rank runs its own replica of
the workload (no collective on the data path) and the slowest rank's time counts.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import shutil
import subprocess
import sys
import tempfile
import time
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Trotter layers/sec at n=1000, chi=4 (mixed vs FP64 GPU) at stated marginal error"
WL = dict(n=1000, seed=0, chi=4, K=3200, dt=0.2, tol=1e-8, max_iter=100)
WORKLOAD_NAME = ("random 3-regular n=1000 (m=1500, 3-colour schedule), J~N(0,1), h~N(0,0.1), "
                 "chi=4, K=3200 layers, dt=0.2, BP tol 1e-8, max 100 sweeps")
# the batched configuration: 256 instances with n uniform over even values in [50, 1000]
BATCH_WL = dict(B=256, seed=0, chi=4, K=400, dt=0.05, tol=1e-8, max_iter=100)
# the precision and bond-dimension sweep: n = 1000 (seed 1), K = 1000, dt = 0.2; layers 1..3
# untimed, layers 4..43 timed
SWEEP_WL = dict(n=1000, seed=1, K=1000, dt=0.2, tol=1e-8, max_iter=100, warm=3, steps=40, chis=(2, 4, 8, 16))
# the scale configuration: n = 100000, chi = 8
SCALE_WL = dict(n=100000, seed=2, chi=8, K=500, dt=0.05, tol=1e-8, max_iter=100, warm=5, steps=10)
SNAPSHOTS = (800, 1600, 2400, 3200)
L2_FLUSH_BYTES = 256 << 20


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gtqa", choices=["gtqa", "reference"])
    p.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64-path comparison run")
    p.add_argument("--no-whole", action="store_true", help="skip the perturbed FP64 anneals of the whole-anneal report")
    p.add_argument("--no-batch", action="store_true", help="skip the batched legs")
    p.add_argument("--no-scale", action="store_true", help="skip the n = 100000, chi = 8 leg")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    p.add_argument("--ncu-scale", type=int, default=None, metavar="N",
                   help="short run of the chi = 8 scale configuration's shape at n = N for ncu: five "
                        "layers, then one gates, one BP (10 sweeps) and one regauge launch")
    p.add_argument("--ncu-case", type=int, default=None, metavar="K0",
                   help="profiling case: anneal layers 1..K0, then one gates launch, one BP launch of 1 sweep "
                        "and, from the same state, one of 21 sweeps (warm start, no regauge); no timing")
    p.add_argument("--budget", type=float, default=20.0, help=argparse.SUPPRESS)
    p.add_argument("--traffic-record", default=None, metavar="CSV",
                   help="no GPU: write the traffic record of the phase kernels from an ncu CSV of "
                        "'--ncu-case 1500' (dram__bytes_read.sum and dram__bytes_write.sum of its gates, two BP and "
                        "regauge launches), tagged with the hash of the current kernel sources")
    p.add_argument("--chi-sweep", action="store_true",
                   help="the precision and bond-dimension sweep (n = 1000, chi in {2, 4, 8, 16}, FP64, mixed "
                        "and complex64, three coupling types): layers/s, BP sweeps and the error against FP64 per cell")
    p.add_argument("--policy-study", action="store_true",
                   help="the regauge policy on the single-instance workload (mixed): R after the gates and "
                        "100 layers with and without a threshold from three points of the anneal")
    p.add_argument("--deg4-study", action="store_true",
                   help="a random 4-regular graph (plain kernels): layers/s, BP sweeps and the mixed and "
                        "complex64 errors against FP64")
    p.add_argument("--bp-study", action="store_true",
                   help="no timing: BP sweeps per layer over the anneal, sweep-by-sweep traces at three late "
                        "layers, and the same anneal with h ~ N(0, 1)")
    a = p.parse_args(argv)
    a.warmup = max(0, a.warmup)
    if a.steps is None:
        a.steps = WL["K"] - a.warmup
    a.steps = max(1, min(a.steps, WL["K"] - a.warmup))
    return a


def sample_layers(W: int, S: int, K: int) -> List[int]:
    """The S timed layers: all of W+1..K when S = K - W, else S layers spread evenly over
    W+1..K (first and last included)."""
    if S >= K - W:
        return list(range(W + 1, K + 1))
    if S == 1:
        return [K]
    return sorted({W + 1 + int(round(i * (K - W - 1) / (S - 1))) for i in range(S)})


def spread(xs: Sequence[int], k: int) -> List[int]:
    """At most k entries of xs, evenly spaced, first and last included."""
    if len(xs) <= k:
        return list(xs)
    return sorted({xs[int(i)] for i in np.linspace(0, len(xs) - 1, k).round()})


def instance():
    from instances import make_instance
    return make_instance(WL["n"], WL["seed"])


def energy(inst, x) -> float:
    """Objective E(x) = sum J_ab x_a x_b + sum h_a x_a of the read-out (the annealer maximises it)."""
    x = np.asarray(x, dtype=np.float64)
    return float(np.sum(inst.J * x[inst.edges[:, 0]] * x[inst.edges[:, 1]]) + np.sum(inst.h * x))


def compare_marginals(rho, sign, rho_ref, sign_ref) -> dict:
    """max / mean |rho - rho_ref| and the sign agreement over the vertices whose reference
    marginal is clear of the read-out tie (|rho00 - 1/2| > 1e-3); null when none is."""
    err = np.abs(rho - rho_ref)
    clear = np.abs(rho_ref[:, 0, 0].real - 0.5) > 1e-3
    agree = float(np.mean(sign[clear] == sign_ref[clear])) if clear.any() else None
    return {"max_abs": float(err.max()), "mean_abs": float(err.mean()), "sign_agreement": agree,
            "clear_vertices": int(clear.sum())}


# ---------------------------------------------------------------------------
# CPU oracle, timed on a bounded sample of the same layers
# ---------------------------------------------------------------------------
def oracle_sampled_rate(steps: Sequence[dict], budget_s: float) -> dict:
    """Layers/s of the CPU oracle on sampled layers of this workload.

    Each step is one layer k from a given state (Gamma, lambda after layer k-1) with that
    layer's BP sweep count s.  A step times a fraction f = q/m of the layer's per-unit work
    with the oracle's own functions: the gates of q edges (in schedule order, from a rotating
    offset), the mixing gate on the matching share of vertices, the symmetric split of the
    touched vertices, s BP message updates of the 2q directed messages of those edges, and the
    per-edge Vidal-gauge step of those edges.  q is sized by a short calibration step so that
    every step takes about budget_s / len(steps) seconds.  The layer's time is estimated as
    t / f, and value = steps / sum of the estimated layer times.
    """
    from oracle import gtqa_oracle as O
    inst = instance()
    n, m = inst.n, inst.m
    order = sorted(range(m), key=lambda e: (int(inst.colour[e]), e))
    per_step = budget_s / max(1, len(steps))

    def one(st, k, s_k, off, q):
        tZ, tX = O.schedule(k, WL["K"], WL["dt"])
        deg = [len(x) for x in st.inc]
        sel = [order[(off + i) % m] for i in range(q)]
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
        for _ in range(max(1, s_k)):
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
        return time.perf_counter() - t0

    est, qs, tot = [], [], 0.0
    for j, sp in enumerate(steps):
        q0 = 4   # calibration on a fresh copy of the state, then the timed step
        tc = one(sp["state"](), sp["k"], sp["sweeps"], 0, q0)
        q = int(min(m, max(1, round(q0 * per_step / max(tc, 1e-6)))))
        t = one(sp["state"](), sp["k"], sp["sweeps"], (j * 97) % m, q)
        est.append(t * m / q)
        qs.append(q)
        tot += t
    return {"value": len(steps) / sum(est), "unit": "layers/s", "cores": 1, "kind": "oracle",
            "seconds": tot, "edges_per_step": qs,
            "layers": [int(sp["k"]) for sp in steps], "sweeps": [int(sp["sweeps"]) for sp in steps]}


def cpu_sample_subprocess(path: str, budget: float) -> dict:
    """Runs the oracle timing in a child process with BLAS threads pinned to 1."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        env.pop(k, None)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-sample", path, "--budget", str(budget)]
    r = subprocess.run(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, timeout=1200)
    if r.returncode != 0:
        return {"value": None, "error": r.stderr.decode(errors="replace")[-400:]}
    return json.loads(r.stdout.decode().strip().splitlines()[-1])


def oracle_sample_main(path: str, budget: float) -> dict:
    """Child-process entry: the sampled layers' states were saved by the FP64 GPU run."""
    from oracle import gtqa_oracle as O
    inst = instance()
    with open(os.path.join(path, "layers.json")) as f:
        meta = json.load(f)
    steps = []
    for k, s_k in zip(meta["layers"], meta["sweeps"]):
        z = np.load(os.path.join(path, f"state_{k}.npz"))
        G_, L_ = z["G"], z["L"]
        steps.append({"k": k, "sweeps": s_k, "state": (lambda G_=G_, L_=L_: O.from_padded(inst.n, inst.edges, G_, L_))})
    r = oracle_sampled_rate(steps, budget)
    r["sample"] = (f"{len(steps)} layers spread over the anneal ({meta['layers'][0]}..{meta['layers'][-1]}), each from "
                   f"the FP64 GPU state after the previous layer with its own BP sweep count "
                   f"(mean {np.mean(meta['sweeps']):.1f}); per layer a fraction of the edges' gates, BP updates of "
                   f"their directed messages, symmetric split, mixing and regauge, scaled to whole layers")
    return r


def oracle_own_states_rate(W: int, layers: Sequence[int], budget: float) -> dict:
    """The reference arm: the oracle anneals layers 1..W itself (no GPU), and every timed step
    is a sampled layer k from that state with the sweep count of the oracle's own layer W."""
    from oracle import gtqa_oracle as O
    inst = instance()
    st = O.plus_state(inst.n, inst.edges)
    s_ref = 1
    for k in range(1, max(W, 1) + 1):
        tZ, tX = O.schedule(k, WL["K"], WL["dt"])
        st, info = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, WL["chi"], WL["tol"], WL["max_iter"])
        s_ref = max(1, int(info["bp_iters"]))
    G_, L_ = O.to_padded(st, 4)
    steps = [{"k": k, "sweeps": s_ref, "state": (lambda: O.from_padded(inst.n, inst.edges, G_, L_))} for k in layers]
    r = oracle_sampled_rate(steps, budget)
    r["sample"] = (f"{max(W, 1)} full oracle layers from |+>, then {len(steps)} steps at the sampled layers "
                   f"{layers[0]}..{layers[-1]} from that state with its BP sweep count ({s_ref}); per step a fraction "
                   f"of the edges' gates, BP updates, symmetric split, mixing and regauge, scaled to whole layers")
    return r


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
# algorithmic and executed work per unit
# ---------------------------------------------------------------------------
def storage_chi(chi: int) -> int:
    return 2 if chi <= 2 else (4 if chi <= 4 else 8)


def gate_flops(chi: int, edges: int, pairs: int, rotations: int, mixed: bool = False):
    """FP64 flops of the simple-update phase as executed (real adds/muls, fma = 2).

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
    flops (the per-message figure of the method; FP32 in the mixed mode)."""
    return float(vertices * 3 * 48 * chi ** 4)


def bp_sweep_flops_executed(chi: int, vertices: int, mixed: bool) -> float:
    """Flops the BP kernel issues per sweep: the mixed kernel contracts the delta form
    (4 contractions, 64 chi^4 per message, FP32); the FP64 kernel the 48 chi^4 of the method."""
    return float(vertices * 3 * (64 if mixed else 48) * chi ** 4)


def _cmac_jacobi(n: int, sweeps: float = 7.5) -> float:
    """Complex MACs of a one-sided Jacobi SVD of order n with vectors: 11 n per pair, n (n - 1) / 2
    pairs per sweep, 7.5 sweeps (the per-unit figure of the method's cost table)."""
    return 11 * n * (n * (n - 1) / 2) * sweeps


def edge_gate_flops(chi: int, mixed: bool) -> Tuple[float, float]:
    """Algorithmic (FP64, FP32) flops of one edge gate with truncation (a2-a3) in the variant that
    runs, from complex MACs of 8 flops: two Householder QRs of the (2 chi^2) x (2 chi) side
    matrices (2 m n^2 - 2/3 n^3 each) and the core M (2 (2 chi)^3), FP64; the one-sided Jacobi SVD
    of order n = 2 chi (FP64, or FP32 sweeps in the mixed mode, which then adds the FP64
    Newton-Schulz step and W = M V, 3 n^3, and two FP64 polish sweeps); the two Q applications (2 chi (m n - n^2 / 2) each; FP32 in the mixed mode);
    and about 50 chi^3 flops of gate and lambda scaling (FP64)."""
    m, n = 2 * chi * chi, 2 * chi
    qr_core = 2 * (2 * m * n * n - 2 * n ** 3 / 3) + 2 * n ** 3
    jac = _cmac_jacobi(n)
    apply_q = 2 * 2 * chi * (m * n - n * n / 2)
    if not mixed:
        return float(8 * (qr_core + jac + apply_q) + 50 * chi ** 3), 0.0
    return float(8 * (qr_core + 3 * n ** 3 + _cmac_jacobi(n, 2.0)) + 50 * chi ** 3), float(8 * (jac + apply_q))


def regauge_edge_flops(chi: int, mixed: bool) -> Tuple[float, float]:
    """Algorithmic (FP64, FP32) flops of the Vidal-gauge step of one edge (a7), from complex MACs:
    two chi x chi Hermitian eigen-decompositions and one chi x chi SVD by one-sided Jacobi (FP64,
    or FP32 sweeps plus the FP64 Newton-Schulz step and two FP64 polish sweeps each, in the mixed
    mode); the square roots
    and inverse square roots (4 chi^3), M (chi^3) and the two transforms X (2 chi^3), FP64; the
    two bond transforms applied to the vertex tensors (2 x 2 chi^4; FP32 in the mixed mode)."""
    n = chi
    jac = 3 * _cmac_jacobi(n)
    fixed = 4 * n ** 3 + n ** 3 + 2 * n ** 3
    apply_g = 2 * 2 * chi ** 4
    if not mixed:
        return float(8 * (jac + fixed + apply_g)), 0.0
    return float(8 * (fixed + 3 * (3 * n ** 3 + _cmac_jacobi(n, 2.0)))), float(8 * (jac + apply_g))


def regauge_flops_executed(chi: int, edges: int, svd_sweeps: int, mixed: bool) -> float:
    """FP64 flops the regauge kernel issues: per counted Jacobi sweep (FP64 sweeps, or the FP64
    polish sweeps of the mixed mode) (N - 1) N / 2 pairs of 14 N + 40 N + 15 flops at N = C;
    per edge the Hermitian parts, roots, M and X (7 C^3 complex MACs), and in the mixed mode the
    three Newton-Schulz steps and products (3 x 3 x 8 C^3)."""
    C = storage_chi(chi)
    per_sweep = (C - 1) * C / 2 * (54 * C + 15)
    fixed = 8 * 7 * C ** 3 + (3 * 3 * 8 * C ** 3 if mixed else 0)
    return float(svd_sweeps * per_sweep + edges * fixed)


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_n1000_chi4.json")
TRAFFIC_SOURCES = [os.path.join(ROOT, "paper_2409_12240_gb300", "csrc", f) for f in ("gtqa_anneal.cuh", "gtqa_common.cuh")]


def kernel_traffic(kernel: str, mixed: bool, chi: int, sweeps_per_launch: float = 0.0):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the committed
    ncu capture of `bench.py --ncu-case`; BP launches are scaled to this run's sweeps per launch
    from the captured 1-sweep and 21-sweep launches.  None if there is no capture for this mode
    or the kernel sources changed since it was taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    r = rec.get("mixed" if mixed else "fp64")
    if not r or r.get("sources_sha256") != sources_sha256() or r.get("chi") != chi or kernel not in r:
        return None
    k = r[kernel]
    if kernel == "bp_kernel":
        return k["fixed_bytes"] + k["bytes_per_sweep"] * sweeps_per_launch
    return k.get("bytes_per_launch")


class Peaks:
    """ALU peaks derived from unit counts and the maximum SM clock (128 FP32 lanes and two FP64
    FMA units per SM, 2 flops per FMA); the FMA microbenchmark is reported beside them."""

    def __init__(self, G, sms: int, mhz: float):
        self.sms, self.mhz = sms, mhz
        self.fp32 = sms * 128 * 2 * mhz * 1e6 / 1e12
        self.fp64 = sms * 2 * 2 * mhz * 1e6 / 1e12
        self.fp64_meas = G.gtqa_alu_peak(True)
        self.fp32_meas = G.gtqa_alu_peak(False)

    def note(self, fp64: bool) -> str:
        lanes, meas = ("2 FP64 FMA units", self.fp64_meas) if fp64 else ("128 FP32 lanes", self.fp32_meas)
        return f"{self.sms} SMs x {lanes} x 2 flop x {self.mhz:.0f} MHz (derived); FMA microbenchmark {meas:.3f} TFLOP/s"


def rooflines(prof: dict, dlt: dict, chi: int, n: int, m: int, mixed: bool, peaks: Peaks, traffic: bool) -> dict:
    """Roofline objects of the three phase kernels from the library's per-launch CUDA events
    (prof: {kernel: (launches, total ms, units)}) and the statistics over the same launches.

    Each kernel's algorithmic work is split by the pipe it runs on in this precision mode (the
    variant that runs): its roofline time is max(F64 / P64, F32 / P32), and `frac` is that time
    over the measured time, reported as achieved / peak of the binding pipe.  The path is
    CUDA-core arithmetic on an L2-resident working set (bound "alu")."""
    out = {}
    C = storage_chi(chi)
    for kname, (nl, ms, units) in prof.items():
        if not nl or kname not in ("gates_kernel", "bp_kernel", "regauge_kernel"):
            continue
        sec = ms * 1e-3
        if kname == "gates_kernel":
            f64u, f32u = edge_gate_flops(chi, mixed)
            f64, f32 = f64u * units, f32u * units
            exe64 = gate_flops(chi, units, int(dlt["svd_pairs"]), int(dlt["svd_rotations"]), mixed)[0]
            unit_count = "edges per launch x the edge gate's algorithmic flops, split by pipe"
            tr = kernel_traffic(kname, mixed, chi) if traffic else None
        elif kname == "bp_kernel":
            sweeps = int(dlt["bp_sweeps"])
            fl = bp_sweep_flops(chi, n, mixed) * sweeps
            norm64 = 20.0 * 3 * n * sweeps   # the FP64 trace reciprocals
            f64, f32 = (norm64, fl) if mixed else (fl + norm64, 0.0)
            exe64 = norm64 if mixed else bp_sweep_flops_executed(C, n, False) * sweeps
            unit_count = "sweeps x 3n directed messages x 48 chi^4 flops (+ the FP64 normalisation)"
            tr = kernel_traffic(kname, mixed, chi, sweeps / nl) if traffic else None
        else:
            f64u, f32u = regauge_edge_flops(chi, mixed)
            f64, f32 = f64u * units, f32u * units
            exe64 = regauge_flops_executed(chi, units, int(dlt["regauge_svd_sweeps"]), mixed)
            unit_count = "edges per launch x the Vidal-gauge step's algorithmic flops, split by pipe"
            tr = kernel_traffic(kname, mixed, chi) if traffic else None
        t64, t32 = f64 / (peaks.fp64 * 1e12), f32 / (peaks.fp32 * 1e12)
        pipe64 = t64 >= t32
        fpipe, peak = (f64, peaks.fp64) if pipe64 else (f32, peaks.fp32)
        ach = fpipe / sec / 1e12
        o = {"kernel": kname, "bound": "alu", "pipe": "fp64" if pipe64 else "fp32", "achieved": ach, "peak": peak,
             "unit": "TFLOP/s", "frac": ach / peak, "traffic": tr, "peak_source": peaks.note(pipe64),
             "algorithmic_fp64_flops_per_launch": f64 / nl, "algorithmic_fp32_flops_per_launch": f32 / nl,
             "roofline_us_per_launch": max(t64, t32) / nl * 1e6, "avg_launch_us": ms / nl * 1e3, "launches": nl,
             "unit_count": unit_count, "executed_fp64_flops_per_launch": exe64 / nl,
             "executed_fp64_frac": exe64 / sec / 1e12 / peaks.fp64}
        if kname == "bp_kernel":
            o["sweeps_per_launch"] = int(dlt["bp_sweeps"]) / nl
            o["us_per_sweep"] = ms * 1e3 / max(int(dlt["bp_sweeps"]), 1)
            o["note"] = ("the working set is L2-resident; each sweep ends in a grid barrier after which the "
                         "neighbours' messages come from L2, so the sweep's latency, not a pipe, bounds it")
        elif kname == "gates_kernel":
            o["note"] = ("algorithmic count: two Householder QRs of the (2 chi^2) x (2 chi) side matrices per edge; "
                         "the kernel factors the four chi^2 x chi blocks of one physical index each (a quarter of "
                         "that QR work), so frac can exceed 1 where the QR dominates (chi = 8); "
                         "executed_fp64_frac is the FP64 work the kernel issues")
        out[kname] = o
    return out


def layer_roofline(roofs: dict) -> dict:
    """The layer's roofline time as the sum of its kernels' roofline times (they run one after
    another), over the measured time of the same launches."""
    t_roof = sum(r["roofline_us_per_launch"] * r["launches"] for r in roofs.values())
    t_meas = sum(r["avg_launch_us"] * r["launches"] for r in roofs.values())
    return {"frac": t_roof / t_meas if t_meas else None, "roofline_us": t_roof, "measured_us": t_meas,
            "note": "sum over the gates, BP and regauge launches of max(F64/P64, F32/P32) per launch"}


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


STAT_KEYS = ("launches", "bp_sweeps", "bp_calls", "bp_not_converged_calls", "svd_pairs", "svd_rotations",
             "bp_exact_passes", "regauge_svd_sweeps")


def walk(G, s, K: int, dt: float, tol: float, mi: int, timed: Sequence[int], stream, flush,
         snaps: Sequence[int] = (), save_before: Sequence[int] = (), profile: bool = False, clocks=None,
         dist=None, state_dir: Optional[str] = None) -> dict:
    """Layers 1..K of one anneal through gtqa_anneal_graph.  Every layer in `timed` is bracketed
    by CUDA events on the library's stream, after an L2 flush that lies outside the events; the
    layers between timed ones run untimed.  With `profile`, the library's per-phase events of
    the timed layers are summed (the roofline's kernel durations).  Returns the timed
    milliseconds, statistics and profile deltas over the timed layers, per-timed-layer sweeps,
    marginals at the snapshot layers, and (into state_dir) the state before given layers."""
    import torch
    timed = sorted(set(int(k) for k in timed))
    tset, sset, bset = set(timed), set(snaps), set(save_before)
    marks = sorted(tset | sset | bset)
    ev = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for k in timed}
    dsum = {k: 0 for k in STAT_KEYS}
    psum: Dict[str, list] = {}
    per_layer = {}
    snap_out = {}
    if profile:
        G.gtqa_profile(s, True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    k = 1
    with torch.cuda.stream(stream):
        for e in marks:
            if e > k:
                G.gtqa_anneal_graph(s, k, e - 1, K, dt, tol, mi)
            if e in bset and state_dir:
                Gm, L, _ = G.gtqa_get_state(s)
                np.savez(os.path.join(state_dir, f"state_{e}.npz"), G=Gm, L=L)
            if e in tset:
                st0 = G.gtqa_stats(s)
                p0 = G.gtqa_profile_read(s) if profile else None
                flush.fill_(e & 0xFF)
                ev[e][0].record(stream)
                G.gtqa_anneal_graph(s, e, e, K, dt, tol, mi)
                ev[e][1].record(stream)
                st1 = G.gtqa_stats(s)
                for key in STAT_KEYS:
                    dsum[key] += st1[key] - st0[key]
                per_layer[e] = {"sweeps": st1["bp_sweeps"] - st0["bp_sweeps"],
                                "max_iter": st1["bp_not_converged_calls"] - st0["bp_not_converged_calls"]}
                if profile:
                    p1 = G.gtqa_profile_read(s)
                    for kn in p1:
                        a0 = psum.setdefault(kn, [0, 0.0, 0])
                        a0[0] += p1[kn][0] - p0[kn][0]
                        a0[1] += p1[kn][1] - p0[kn][1]
                        a0[2] += p1[kn][2] - p0[kn][2]
            else:
                G.gtqa_anneal_graph(s, e, e, K, dt, tol, mi)
            if e in sset:
                snap_out[e] = G.gtqa_marginals(s)
            k = e + 1
        if k <= K:
            G.gtqa_anneal_graph(s, k, K, K, dt, tol, mi)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ck = clocks.stop() if clocks else None
    if profile:
        G.gtqa_profile(s, False)
    t_ms = float(sum(ev[k][0].elapsed_time(ev[k][1]) for k in timed))
    rho, sign = G.gtqa_marginals(s)
    return {"t_ms": t_ms, "stats": dsum, "prof": {kn: tuple(v) for kn, v in psum.items()}, "per_layer": per_layer,
            "snaps": snap_out, "rho": rho, "sign": sign, "clocks": ck}


KERNELS = ("gates_kernel", "bp_kernel", "regauge_kernel")


def tune_launch(G, make_state, K: int, dt: float, tol: float, mi: int, k_tune: int) -> dict:
    """gtqa_autotune on a separate state annealed (untimed) through layers 1..k_tune-1 of the
    workload, timing layer k_tune; returns the launch table it picks (per kernel: grid,
    shape variant, threads per block, team) and the time the search took."""
    s = make_state()
    try:
        if k_tune > 1:
            G.gtqa_anneal_graph(s, 1, k_tune - 1, K, dt, tol, mi)
        t0 = time.perf_counter()
        G.gtqa_autotune(s, k_tune / K, dt, tol, mi)
        t_s = time.perf_counter() - t0
        table = G.gtqa_launch_shape(s)
    finally:
        G.gtqa_destroy(s)
    return {"table": table, "tuned_at_layer": k_tune, "search_s": round(t_s, 3)}


def apply_launch(G, s, tuned: dict) -> None:
    t = tuned["table"]
    G.gtqa_set_shape(s, [t[k]["variant"] for k in KERNELS])
    G.gtqa_set_grid(s, [t[k]["grid"] for k in KERNELS])


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
    W, S = a.warmup, a.steps
    Ks, dt, tol, mi, chi = WL["K"], WL["dt"], WL["tol"], WL["max_iter"], WL["chi"]
    timed = sample_layers(W, S, Ks)
    S = len(timed)
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    props = torch.cuda.get_device_properties(local)

    def make(p, J=None, inst_=None):
        x = inst_ or inst
        return G.gtqa_create(x.n, x.edges, x.J if J is None else J, x.h, chi, x.colour,
                             G.gtqa_options_init(precision=p, cuda_stream=stream.cuda_stream))

    # ---- launch shapes: gtqa_autotune from the state before the middle layer of the anneal ----
    tuned = tune_launch(G, lambda: make(prec), Ks, dt, tol, mi, Ks // 2)

    # ---- the timed run of the chosen precision ----
    clocks = Clocks(local)
    s = make(prec)
    apply_launch(G, s, tuned)
    main = walk(G, s, Ks, dt, tol, mi, timed, stream, flush, snaps=SNAPSHOTS, profile=True, clocks=clocks, dist=dist)
    G.gtqa_destroy(s)
    t_ms, value = replica_throughput(main["t_ms"], S, world, dist, "cuda")
    ck = main["clocks"]
    mhz = (ck or {}).get("sm_max_mhz") or 2070.0
    peaks = Peaks(G, props.multi_processor_count, mhz)
    roofs = rooflines(main["prof"], main["stats"], chi, inst.n, inst.m, mixed, peaks, traffic=True)
    total_prof = sum(v[1] for v in main["prof"].values())
    dom = max(roofs, key=lambda kn: main["prof"][kn][1])
    kernel_share = {kn: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / total_prof, 4) if total_prof else 0}
                    for kn, v in main["prof"].items() if v[0]}

    # ---- the FP64 path on the same layers; its states before a few sampled layers feed the
    # per-layer error and the CPU baseline ----
    err_layers = spread(timed, 6)
    cpu_layers = spread(timed, 20)
    state_dir = tempfile.mkdtemp(prefix="gtqa_bench_")
    fp64 = None
    whole = None
    cpu = None
    try:
        run64 = None
        if mixed and not a.no_fp64:
            tuned64 = tune_launch(G, lambda: make(G.GTQA_FP64), Ks, dt, tol, mi, Ks // 2)
            s = make(G.GTQA_FP64)
            apply_launch(G, s, tuned64)
            run64 = walk(G, s, Ks, dt, tol, mi, timed, stream, flush, snaps=SNAPSHOTS,
                         save_before=sorted(set(err_layers) | set(cpu_layers)), profile=True, state_dir=state_dir)
            G.gtqa_destroy(s)
            r64 = rooflines(run64["prof"], run64["stats"], chi, inst.n, inst.m, False, peaks, traffic=True)
            per = per_layer_error(G, make, err_layers, state_dir)
            fp64 = {"value": world * S / (run64["t_ms"] / 1e3), "unit": "layers/s", "ms_per_step": run64["t_ms"] / S,
                    "bp_sweeps_per_layer": run64["stats"]["bp_sweeps"] / S,
                    "bp_layers_at_max_iter": run64["stats"]["bp_not_converged_calls"] / S,
                    "speedup_mixed_over_fp64": run64["t_ms"] / main["t_ms"],
                    "marginal_error_per_layer": per, "roofline": r64, "layer_roofline": layer_roofline(r64),
                    "launch": tuned64, "note": "the same timed layers on the FP64 path"}
            if not a.no_whole:
                whole = whole_anneal(G, make, inst, main, run64, stream, flush, props.multi_processor_count, tuned64)
        if rank == 0 and world == 1 and not a.no_cpu and run64 is not None:
            with open(os.path.join(state_dir, "layers.json"), "w") as f:
                json.dump({"layers": cpu_layers, "sweeps": [int(run64["per_layer"][k]["sweeps"]) for k in cpu_layers]}, f)
            cpu = cpu_sample_subprocess(state_dir, a.budget)
    finally:
        shutil.rmtree(state_dir, ignore_errors=True)

    # ---- end to end through the public API with host buffers: the whole anneal ----
    e2e = None
    if not a.no_e2e:
        rho_h = torch.empty((inst.n, 2, 2), dtype=torch.complex128, pin_memory=True).numpy()
        sign_h = torch.empty(inst.n, dtype=torch.int8, pin_memory=True).numpy()
        h2d = inst.edges.nbytes + inst.J.nbytes + inst.h.nbytes + inst.colour.nbytes
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s3 = make(prec)
        apply_launch(G, s3, tuned)
        for k in range(1, Ks + 1):
            G.gtqa_anneal_graph(s3, k, k, Ks, dt, tol, mi)
            G.gtqa_marginals(s3, rho_h, sign_h)
        G.gtqa_destroy(s3)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        e2e = {"value": world * Ks / t_e2e, "unit": "layers/s", "h2d_bytes_per_step": h2d / Ks,
               "d2h_bytes_per_step": rho_h.nbytes + sign_h.nbytes,
               "note": "create from host arrays, every layer 1..K (CUDA-graph replay) followed by the marginals "
                       "and read-out into pinned host buffers, destroy; wall clock"}

    batch = None if a.no_batch else batched_legs(G, stream, flush, peaks, W, S, fp64)
    scale = None if a.no_scale else scale_leg(G, stream, flush, peaks, fp64)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    nl = S
    out = {
        "metric": METRIC, "value": value, "unit": "layers/s", "n_gpus": world, "steps": S, "warmup": W,
        "ms_per_step": t_ms / S, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64/f64" if mixed else "c128/f64", "data": "synthetic",
        "config": config_dict(a, timed, world),
        "bp_sweeps_per_layer": main["stats"]["bp_sweeps"] / nl,
        "bp_layers_at_max_iter": main["stats"]["bp_not_converged_calls"] / nl,
        "bp_exact_passes": main["stats"]["bp_exact_passes"],
        "launch": tuned, "fp64_path": fp64, "whole_anneal": whole,
        "roofline": roofs[dom], "roofline_other_kernels": {k: v for k, v in roofs.items() if k != dom},
        "layer_roofline": layer_roofline(roofs), "kernel_share": kernel_share,
        "alu_peaks_tflops": {"fp32": peaks.fp32, "fp64": peaks.fp64, "fp32_measured": peaks.fp32_meas,
                             "fp64_measured": peaks.fp64_meas},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(main["stats"]["launches"]), "clocks": ck,
        "batched": batch, "scale": scale,
        "final_marginals": {"mean_abs_z": float(np.mean(np.abs(main["rho"][:, 0, 0].real - main["rho"][:, 1, 1].real))),
                            "E": energy(inst, main["sign"])},
    }
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def config_dict(a, timed, world) -> dict:
    return {"workload": WORKLOAD_NAME, "precision": a.precision,
            "layers_timed": {"count": len(timed), "first": timed[0], "last": timed[-1],
                             "spread": len(timed) < WL["K"] - a.warmup},
            "l2": "flushed before every timed layer (256 MiB write, outside the timed events)",
            "launch": "one CUDA-graph replay per layer (gates, BP, regauge)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def per_layer_error(G, make, layers: Sequence[int], state_dir: str) -> dict:
    """Marginal error introduced by one mixed-precision layer: at the given layers k the FP64
    state after layer k-1 is loaded into a mixed and an FP64 state, layer k runs in both, and
    max |rho_mixed - rho_fp64| over vertices is recorded with the sign agreement."""
    Ks, dt, tol, mi = WL["K"], WL["dt"], WL["tol"], WL["max_iter"]
    out = {}
    for k in layers:
        z = np.load(os.path.join(state_dir, f"state_{k}.npz"))
        res = []
        for p in (G.GTQA_MIXED, G.GTQA_FP64):
            s = make(p)
            n_, m_, C_, _ = G.gtqa_sizes(s)
            G.gtqa_set_state(s, z["G"], z["L"], np.zeros((2 * m_, C_, C_), dtype=np.complex128))
            G.gtqa_anneal(s, k, k, Ks, dt, tol, mi)
            res.append(G.gtqa_marginals(s))
            G.gtqa_destroy(s)
        (rm, sm_), (rf, sf) = res
        out[str(k)] = compare_marginals(rm, sm_, rf, sf)
    agrees = [v["sign_agreement"] for v in out.values() if v["sign_agreement"] is not None]
    return {"max_abs": max(v["max_abs"] for v in out.values()),
            "min_sign_agreement": min(agrees) if agrees else None, "samples": out,
            "note": "one layer in each mode from the same FP64 state at layer k-1"}


def whole_anneal(G, make, inst, main, run64, stream, flush, sms: int, tuned64: dict) -> dict:
    """The read-out over the whole anneal: the mixed run and FP64 runs whose inputs differ at
    rounding level (every J_ab moved by one ulp; every J_ab scaled by 1 + 2^-24 xi with seeded
    signs xi, the size of complex64 rounding; another grid size of the persistent kernels,
    which reorders nothing and must give identical results), each against the FP64 run at
    layers 800, 1600, 2400 and 3200, with the objective E(x) of each final read-out."""
    Ks, dt, tol, mi = WL["K"], WL["dt"], WL["tol"], WL["max_iter"]
    rng = np.random.default_rng(2409122400 + 77)
    runs = {"fp64_J_plus_1ulp": dict(J=np.nextafter(inst.J, np.inf)),
            "fp64_J_rel_2^-24": dict(J=inst.J * (1.0 + 2.0 ** -24 * rng.choice([-1.0, 1.0], size=inst.m))),
            "fp64_grid_7/8": dict(grid=max(1, sms * 7 // 8))}
    snaps = {"mixed": main["snaps"], "fp64": run64["snaps"]}
    finals = {"mixed": main["sign"], "fp64": run64["sign"]}
    for name, kw in runs.items():
        s = make(G.GTQA_FP64, J=kw.get("J"))
        apply_launch(G, s, tuned64)   # the FP64 run's launch shapes
        if "grid" in kw:
            G.gtqa_set_grid(s, [kw["grid"]] * 3)
        r = walk(G, s, Ks, dt, tol, mi, [], stream, flush, snaps=SNAPSHOTS)
        G.gtqa_destroy(s)
        snaps[name] = r["snaps"]
        finals[name] = r["sign"]
    out = {"reference": "fp64", "E_fp64": energy(inst, finals["fp64"]), "runs": {}}
    for name in snaps:
        if name == "fp64":
            continue
        d = {"E": energy(inst, finals[name])}
        for k in SNAPSHOTS:
            rho, sg = snaps[name][k]
            rf, sf = snaps["fp64"][k]
            d[str(k)] = compare_marginals(rho, sg, rf, sf)
        out["runs"][name] = d
    Es = [out["E_fp64"]] + [v["E"] for k, v in out["runs"].items() if k.startswith("fp64")]
    out["fp64_E_range"] = [min(Es), max(Es)]
    out["mixed_E_within_fp64_range"] = bool(min(Es) <= out["runs"]["mixed"]["E"] <= max(Es))
    out["note"] = ("BP reaches max_iter without converging in most late-anneal layers; there the state follows an "
                   "unstable map, so the read-out depends on rounding-level differences of the inputs")
    return out


def batched_legs(G, stream, flush, peaks: Peaks, W: int, S: int, fp64) -> dict:
    """Mixed batched throughput, instance-layers/s, with the FP64 single-instance rate beside it:
    (a) 16 seeded n = 1000 instances of the single-instance workload's shape in one batched
    state; (b) the batched configuration (256 instances, n uniform over even values in
    [50, 1000], K = 400, dt = 0.05).  Both anneal through CUDA-graph replays with S timed layers
    spread over the anneal as in the main run."""
    from instances import make_batch, make_instance
    out = {}
    legs = {"16x_n1000": ([make_instance(1000, s_) for s_ in range(16)], WL["K"], WL["dt"], WL["tol"], WL["max_iter"]),
            "256_uneven": (make_batch(BATCH_WL["B"], seed=BATCH_WL["seed"]), BATCH_WL["K"], BATCH_WL["dt"],
                           BATCH_WL["tol"], BATCH_WL["max_iter"])}
    for name, (insts, K, dt, tol, mi) in legs.items():
        def mk():
            return G.gtqa_create_batch([x.n for x in insts], [x.edges for x in insts], [x.J for x in insts],
                                       [x.h for x in insts], 4, [x.colour for x in insts],
                                       G.gtqa_options_init(precision=G.GTQA_MIXED, cuda_stream=stream.cuda_stream))
        w0 = min(W, K - 1)
        tuned = tune_launch(G, mk, K, dt, tol, mi, w0 + 1)
        s = mk()
        apply_launch(G, s, tuned)
        timed = sample_layers(w0, min(S, K - w0), K)
        r = walk(G, s, K, dt, tol, mi, timed, stream, flush, profile=True)
        G.gtqa_destroy(s)
        N = sum(x.n for x in insts)
        M = sum(x.m for x in insts)
        roofs = rooflines(r["prof"], r["stats"], 4, N, M, True, peaks, traffic=False)
        dom = max(roofs, key=lambda kn: r["prof"][kn][1])
        L = len(timed)
        out[name] = {"instances": len(insts), "vertices": N, "edges": M, "K": K, "dt": dt,
                     "layers_timed": {"count": L, "first": timed[0], "last": timed[-1]},
                     "instance_layers_per_s": len(insts) * L / (r["t_ms"] / 1e3),
                     "batch_layers_per_s": L / (r["t_ms"] / 1e3), "ms_per_layer": r["t_ms"] / L,
                     "bp_sweeps_per_layer": r["stats"]["bp_sweeps"] / L,
                     "fp64_single_instance_layers_per_s": (fp64 or {}).get("value"), "launch": tuned,
                     "roofline": roofs[dom], "roofline_other_kernels": {k: v for k, v in roofs.items() if k != dom},
                     "layer_roofline": layer_roofline(roofs)}
    return out


def scale_leg(G, stream, flush, peaks: Peaks, fp64) -> dict:
    """The scale configuration (n = 100000, m = 150000, chi = 8, mixed, K = 500, dt = 0.05),
    HBM-resident: layers 1..5 untimed, layers 6..15 timed (the whole anneal takes minutes)."""
    from instances import make_instance
    w = SCALE_WL
    inst = make_instance(w["n"], w["seed"])

    def mk():
        return G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, w["chi"], inst.colour,
                             G.gtqa_options_init(precision=G.GTQA_MIXED, cuda_stream=stream.cuda_stream))
    s = mk()
    timed = list(range(w["warm"] + 1, w["warm"] + w["steps"] + 1))
    G.gtqa_anneal_graph(s, 1, w["warm"], w["K"], w["dt"], w["tol"], w["max_iter"])
    # gtqa_autotune on this state, timing the first timed layer (it restores the state)
    t0 = time.perf_counter()
    G.gtqa_autotune(s, timed[0] / w["K"], w["dt"], w["tol"], w["max_iter"])
    tuned = {"table": G.gtqa_launch_shape(s), "tuned_at_layer": timed[0],
             "search_s": round(time.perf_counter() - t0, 3)}
    r = walk_range(G, s, w, timed, stream, flush)
    G.gtqa_destroy(s)
    roofs = rooflines(r["prof"], r["stats"], w["chi"], inst.n, inst.m, True, peaks, traffic=False)
    dom = max(roofs, key=lambda kn: r["prof"][kn][1])
    L = len(timed)
    return {"n": inst.n, "m": inst.m, "chi": w["chi"], "K": w["K"], "dt": w["dt"], "launch": tuned,
            "layers_timed": {"count": L, "first": timed[0], "last": timed[-1]},
            "layers_per_s": L / (r["t_ms"] / 1e3), "ms_per_layer": r["t_ms"] / L,
            "bp_sweeps_per_layer": r["stats"]["bp_sweeps"] / L,
            "roofline": roofs[dom], "roofline_other_kernels": {k: v for k, v in roofs.items() if k != dom},
            "layer_roofline": layer_roofline(roofs)}


def walk_range(G, s, w, timed, stream, flush) -> dict:
    """Times consecutive layers `timed` (already annealed up to timed[0] - 1) with per-layer
    CUDA events and the library's per-phase events."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in timed]
    G.gtqa_profile(s, True)
    st0 = G.gtqa_stats(s)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for j, k in enumerate(timed):
            flush.fill_(k & 0xFF)
            ev[j][0].record(stream)
            G.gtqa_anneal_graph(s, k, k, w["K"], w["dt"], w["tol"], w["max_iter"])
            ev[j][1].record(stream)
    torch.cuda.synchronize()
    prof = G.gtqa_profile_read(s)
    st1 = G.gtqa_stats(s)
    G.gtqa_profile(s, False)
    return {"t_ms": float(sum(e0.elapsed_time(e1) for e0, e1 in ev)), "prof": prof,
            "stats": {k: st1[k] - st0[k] for k in STAT_KEYS}}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    W = a.warmup
    timed = sample_layers(W, a.steps, WL["K"])
    r = oracle_own_states_rate(W, timed, budget=120.0)
    out = {"impl": "reference", "metric": METRIC, "value": r["value"], "unit": "layers/s", "n_gpus": world,
           "steps": len(timed), "warmup": W, "ms_per_step": 1e3 / r["value"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "c128/f64", "data": "synthetic",
           "config": config_dict(a, timed, world),
           "cpu_baseline": {"value": r["value"], "unit": "layers/s", "cores": 1, "kind": "oracle", "sample": r["sample"]},
           "e2e": {"value": r["value"], "unit": "layers/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
def ncu_case(a):
    """A short run for ncu captures: the launches of interest come after 3 K0 warm-up launches
    (gates, BP, regauge per layer); the gates launch is the (K0+1)-th gates_kernel, the two BP
    launches the (K0+1)-th and (K0+2)-th bp_kernel, the regauge launch the (K0+1)-th
    regauge_kernel."""
    from paper_2409_12240_gb300 import gtqa as G
    G.load(build_if_missing=True)
    inst = instance()
    prec = G.GTQA_MIXED if a.precision == "mixed" else G.GTQA_FP64
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, WL["chi"], inst.colour, G.gtqa_options_init(precision=prec))
    try:
        # the launch shapes gtqa_autotune picks for this workload in the mixed mode (gates in
        # 256-thread blocks, BP and regauge in their default shapes)
        if a.precision == "mixed":
            G.gtqa_set_shape(s, (1, 0, 0))
        K0 = a.ncu_case
        if K0 > 0:
            G.gtqa_anneal(s, 1, K0, WL["K"], WL["dt"], WL["tol"], WL["max_iter"])
        G.gtqa_trotter_layer(s, (K0 + 1) / WL["K"], WL["dt"])
        Gm, L, M = G.gtqa_get_state(s)
        G.gtqa_bp_sweep(s, 0.0, 1, G.GTQA_BP_WARM_START)
        G.gtqa_set_state(s, Gm, L, M)
        G.gtqa_bp_sweep(s, 0.0, 21, G.GTQA_BP_WARM_START)
        G.gtqa_regauge(s)
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
        # the launch shapes gtqa_autotune picks at this shape (512-thread blocks for all three kernels)
        G.gtqa_set_shape(s, (1, 1, 1))
        G.gtqa_anneal(s, 1, 5, K, dt, tol, mi)
        G.gtqa_trotter_layer(s, 6 / K, dt)
        G.gtqa_bp_sweep(s, 0.0, 10, G.GTQA_BP_WARM_START)
        G.gtqa_regauge(s)
        G.gtqa_marginals(s)
    finally:
        G.gtqa_destroy(s)
    print(json.dumps({"ncu_scale": a.ncu_scale, "chi": 8, "precision": "mixed"}))


def bp_study(a):
    """How flooding BP behaves over the single-instance anneal (no timing): per layer the sweeps
    of the FP64 path and whether they reached max_iter; at three late layers the distance of
    every sweep of a 160-sweep run from the warm start, with the change of each message between
    consecutive sweeps (d1) and two sweeps apart (d2): a period-2 oscillation gives d2 << d1, a
    steady drift d2 ~ 2 d1.  The same anneal with the fields of the paper's QUBO runs,
    h ~ N(0, 1), is run beside it in FP64 and mixed, with the objective of each read-out."""
    from instances import make_instance
    from paper_2409_12240_gb300 import gtqa as G
    G.load(build_if_missing=True)
    K, dt, tol, mi, chi = WL["K"], WL["dt"], WL["tol"], WL["max_iter"], WL["chi"]
    out = {}
    for hname, hs in (("h_std_0.1", 0.1), ("h_std_1", 1.0)):
        inst = make_instance(WL["n"], WL["seed"], h_std=hs)
        res = {}
        for pname, prec in (("fp64", G.GTQA_FP64), ("mixed", G.GTQA_MIXED)):
            s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour, G.gtqa_options_init(precision=prec))
            sweeps, maxit, states = [], [], {}
            prev = G.gtqa_stats(s)
            for k in range(1, K + 1):
                if hs == 0.1 and prec == G.GTQA_FP64 and k in (1501, 2001, 2801):
                    states[k] = G.gtqa_get_state(s)
                G.gtqa_anneal_graph(s, k, k, K, dt, tol, mi)
                st = G.gtqa_stats(s)
                sweeps.append(st["bp_sweeps"] - prev["bp_sweeps"])
                maxit.append(st["bp_not_converged_calls"] - prev["bp_not_converged_calls"])
                prev = st
            rho, sign = G.gtqa_marginals(s)
            G.gtqa_destroy(s)
            sw = np.array(sweeps)
            first = int(np.argmax(np.array(maxit) > 0)) + 1 if any(maxit) else None
            res[pname] = {"mean_sweeps": float(sw.mean()), "layers_at_max_iter": float(np.mean(maxit)),
                          "first_max_iter_layer": first,
                          "sweeps_per_100_layers": [float(x) for x in sw.reshape(-1, 100).mean(axis=1)],
                          "histogram": {"bins": [1, 2, 3, 5, 10, 20, 50, 100, 101],
                                        "counts": np.histogram(sw, bins=[1, 2, 3, 5, 10, 20, 50, 100, 101])[0].tolist()},
                          "E": energy(inst, sign), "sign": sign}
            if states:
                traces = {}
                for k, (Gm, L, Mg) in states.items():
                    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour)
                    G.gtqa_set_state(s, Gm, L, Mg)
                    G.gtqa_trotter_layer(s, k / K, dt)
                    dists, ms = [], []
                    for t in range(160):
                        _, d, _ = G.gtqa_bp_sweep(s, 0.0, 1, G.GTQA_BP_WARM_START if t == 0 else 0)
                        dists.append(d)
                        ms.append(G.gtqa_get_state(s)[2])
                    G.gtqa_destroy(s)
                    ms = np.array(ms)
                    d1 = np.linalg.norm(ms[1:] - ms[:-1], axis=(2, 3)).sum(axis=1)
                    d2 = np.linalg.norm(ms[2:] - ms[:-2], axis=(2, 3)).sum(axis=1)
                    moving = (np.linalg.norm(ms[-1] - ms[-2], axis=(1, 2)) > 1e-6).mean()
                    traces[str(k)] = {"dist_per_sweep": [float(dists[i]) for i in (0, 1, 2, 5, 10, 20, 50, 100, 159)],
                                      "dist_min_max_last_100": [float(min(dists[60:])), float(max(dists[60:]))],
                                      "d2_over_d1_last_50": float(np.mean(d2[-50:] / d1[-50:])),
                                      "messages_moving_last_sweep": float(moving)}
                res["fp64_traces"] = traces
        res["sign_agreement_mixed_fp64"] = float(np.mean(res["mixed"].pop("sign") == res["fp64"].pop("sign")))
        out[hname] = res
    print(json.dumps({"bp_study": out, "workload": WORKLOAD_NAME}))


def chi_sweep(a):
    """The precision and bond-dimension sweep.  Three coupling types on the same seeded graph
    (J = +1 with h = 0, J = -1 with h = 0 (the MaxCut couplings of Sec. IV A), and J ~ N(0, 1)
    with h ~ N(0, 0.1)), chi in {2, 4, 8, 16}, each in the FP64, mixed and complex64 modes, with
    the default launch shapes.  Layers 1..3 run untimed.  Layers 4..43 are then timed one by one
    with CUDA events on the library's stream (gtqa_anneal, one layer per call), each after an
    L2 flush outside the events.  Each cell reports layers/s and BP sweeps per layer over the
    timed layers.  It also reports max / mean |rho - rho_FP64| per vertex after layer 43, against
    the FP64 cell of the same couplings and chi (the FP64 path agrees with the oracle to 1e-10),
    and the sign agreement over the clear vertices (none for the Z2-symmetric h = 0 couplings)."""
    import torch
    from instances import make_instance
    from paper_2409_12240_gb300 import gtqa as G
    G.load(build_if_missing=True)
    w = SWEEP_WL
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    timed = list(range(w["warm"] + 1, w["warm"] + w["steps"] + 1))
    modes = (("fp64", G.GTQA_FP64), ("mixed", G.GTQA_MIXED), ("complex64", G.GTQA_C64))
    out = {}
    for cname, J, hs in (("J=+1,h=0", "ferro", 0.0), ("J=-1,h=0 (MaxCut)", "maxcut", 0.0),
                         ("J~N(0,1),h~N(0,0.1)", "gauss", 0.1)):
        inst = make_instance(w["n"], w["seed"], J=J, h_std=hs)
        cells = {}
        for chi in w["chis"]:
            row, ref = {}, None
            for mname, prec in modes:
                s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour,
                                  G.gtqa_options_init(precision=prec, cuda_stream=stream.cuda_stream))
                try:
                    G.gtqa_anneal(s, 1, w["warm"], w["K"], w["dt"], w["tol"], w["max_iter"])
                    t_ms, st0, st1 = timed_layers(
                        G, s, timed, lambda s_, k: G.gtqa_anneal(s_, k, k, w["K"], w["dt"], w["tol"], w["max_iter"]),
                        stream, flush)
                    rho, sign = G.gtqa_marginals(s)
                finally:
                    G.gtqa_destroy(s)
                cell = {"layers_per_s": len(timed) / (t_ms / 1e3),
                        "bp_sweeps_per_layer": (st1["bp_sweeps"] - st0["bp_sweeps"]) / len(timed)}
                if ref is None:
                    ref = (rho, sign)
                else:
                    cell.update(compare_marginals(rho, sign, *ref))
                row[mname] = cell
            cells[str(chi)] = row
        out[cname] = cells
    print(json.dumps({"chi_sweep": out, "n": w["n"], "seed": w["seed"], "K": w["K"], "dt": w["dt"], "tol": w["tol"],
                      "max_iter": w["max_iter"], "layers_timed": {"first": timed[0], "last": timed[-1]},
                      "error_reference": "the FP64 cell of the same couplings and chi, after the last timed layer"}))


def timed_layers(G, s, layers: Sequence[int], run, stream, flush) -> Tuple[float, dict, dict]:
    """Runs run(s, k) for each layer k, each bracketed by CUDA events on the library's stream
    after an L2 flush outside the events; returns the summed time (ms) and the statistics
    before and after."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in layers]
    torch.cuda.synchronize()
    st0 = G.gtqa_stats(s)
    with torch.cuda.stream(stream):
        for j, k in enumerate(layers):
            flush.fill_(k & 0xFF)
            ev[j][0].record(stream)
            run(s, k)
            ev[j][1].record(stream)
    torch.cuda.synchronize()
    st1 = G.gtqa_stats(s)
    return float(sum(e0.elapsed_time(e1) for e0, e1 in ev)), st0, st1


POLICY_WL = dict(starts=(300, 1500, 2800), layers=100, threshold=1e-2)


def policy_study(a):
    """The regauge policy (Sec. II C: regauge only when the residual R of App. C is large) on the
    single-instance workload in the mixed mode.  The mixed path anneals layers 1..k0-1 for
    k0 in {300, 1500, 2800}.  From each of these states: R after the gates of layer k0; layers
    k0..k0+99 with the regauge in every layer; the same layers through gtqa_anneal_policy with
    R threshold 1e-2.  Each run reports layers/s (per-layer CUDA events after an L2 flush) and
    the regauged and skipped counts.  The policy run also reports its marginals against the
    every-layer run after the last layer."""
    import torch
    from paper_2409_12240_gb300 import gtqa as G
    G.load(build_if_missing=True)
    K, dt, tol, mi, chi = WL["K"], WL["dt"], WL["tol"], WL["max_iter"], WL["chi"]
    inst = instance()
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def make():
        return G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour,
                             G.gtqa_options_init(precision=G.GTQA_MIXED, cuda_stream=stream.cuda_stream))
    s = make()
    states, k_done = {}, 0
    for k0 in POLICY_WL["starts"]:
        G.gtqa_anneal_graph(s, k_done + 1, k0 - 1, K, dt, tol, mi)
        k_done = k0 - 1
        states[k0] = G.gtqa_get_state(s)
    G.gtqa_destroy(s)
    thr = POLICY_WL["threshold"]
    out = {}
    for k0, st in states.items():
        layers = list(range(k0, k0 + POLICY_WL["layers"]))
        res = {}
        s = make()
        G.gtqa_set_state(s, *st)
        G.gtqa_trotter_layer(s, k0 / K, dt)
        res["R_after_gates"] = G.gtqa_residual(s)
        G.gtqa_destroy(s)
        rho = {}
        for name, run in (("every_layer", lambda s_, k: G.gtqa_anneal(s_, k, k, K, dt, tol, mi)),
                          (f"threshold_{thr:g}", lambda s_, k: G.gtqa_anneal_policy(s_, k, k, K, dt, tol, mi, thr))):
            s = make()
            try:
                G.gtqa_set_state(s, *st)
                r0 = G.gtqa_regauge_counts(s)
                t_ms, st0, st1 = timed_layers(G, s, layers, run, stream, flush)
                r1 = G.gtqa_regauge_counts(s)
                rho[name] = G.gtqa_marginals(s)
            finally:
                G.gtqa_destroy(s)
            cell = {"layers_per_s": len(layers) / (t_ms / 1e3),
                    "bp_sweeps_per_layer": (st1["bp_sweeps"] - st0["bp_sweeps"]) / len(layers)}
            if name != "every_layer":
                cell.update({"regauged": r1[0] - r0[0], "skipped": r1[1] - r0[1]})
                cell["against_every_layer"] = compare_marginals(*rho[name], *rho["every_layer"])
            res[name] = cell
        out[str(k0)] = res
    print(json.dumps({"policy_study": out, "workload": WORKLOAD_NAME, "precision": "mixed",
                      "layers_per_start": POLICY_WL["layers"], "threshold": thr}))


DEG4_WL = dict(n=200, seed=0, chi=4, K=20, dt=0.3, tol=1e-10, max_iter=100, warm=1, steps=11)


def deg4_study(a):
    """A seeded random 4-regular graph (Sec. V), n = 200, J ~ N(0, 1), h ~ N(0, 0.1), chi = 4,
    K = 20, dt = 0.3, BP tol 1e-10, on the plain kernels.  Layer 1 runs untimed; layers 2..12
    are timed one by one (CUDA events after an L2 flush).  Per precision mode: layers/s, BP
    sweeps per layer, and for the mixed and complex64 modes max / mean |rho - rho_FP64| after
    layer 12 with the sign agreement over clear vertices."""
    import torch
    from instances import make_instance
    from paper_2409_12240_gb300 import gtqa as G
    G.load(build_if_missing=True)
    w = DEG4_WL
    inst = make_instance(w["n"], w["seed"], d=4)
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    layers = list(range(w["warm"] + 1, w["warm"] + w["steps"] + 1))
    out, ref = {}, None
    for mname, prec in (("fp64", G.GTQA_FP64), ("mixed", G.GTQA_MIXED), ("complex64", G.GTQA_C64)):
        s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, w["chi"], inst.colour,
                          G.gtqa_options_init(precision=prec, cuda_stream=stream.cuda_stream))
        try:
            G.gtqa_anneal(s, 1, w["warm"], w["K"], w["dt"], w["tol"], w["max_iter"])
            t_ms, st0, st1 = timed_layers(
                G, s, layers, lambda s_, k: G.gtqa_anneal(s_, k, k, w["K"], w["dt"], w["tol"], w["max_iter"]),
                stream, flush)
            rho, sign = G.gtqa_marginals(s)
        finally:
            G.gtqa_destroy(s)
        cell = {"layers_per_s": len(layers) / (t_ms / 1e3),
                "bp_sweeps_per_layer": (st1["bp_sweeps"] - st0["bp_sweeps"]) / len(layers)}
        if ref is None:
            ref = (rho, sign)
        else:
            cell.update(compare_marginals(rho, sign, *ref))
        out[mname] = cell
    print(json.dumps({"deg4_study": out, **{k: w[k] for k in ("n", "seed", "chi", "K", "dt", "tol", "max_iter")},
                      "layers_timed": {"first": layers[0], "last": layers[-1]}}))


TRAFFIC_CASE = 1500
TRAFFIC_NCU = ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none "
               "-k regex:\"gates_kernel|bp_kernel|regauge_kernel\" -s 4500 -c 4 --csv --log-file traffic.csv "
               f"python bench.py --ncu-case {TRAFFIC_CASE}")


def sources_sha256() -> str:
    h = hashlib.sha256()
    for p in TRAFFIC_SOURCES:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traffic_record(path: str) -> dict:
    """Reads the ncu CSV of the four captured launches of `--ncu-case 1500` (mixed: the gates
    launch of layer 1501, BP launches of 1 and 21 sweeps from the same state, the regauge) and
    writes the per-launch DRAM bytes to the traffic record with the hash of the kernel sources.
    The BP launch's bytes are split into a fixed part and a part per sweep."""
    import csv
    with open(path, newline="") as f:
        rows = list(csv.reader(f))
    head = next(i for i, r in enumerate(rows) if r and r[0] == "ID")
    cols = {name: j for j, name in enumerate(rows[head])}
    launches: Dict[int, dict] = {}
    for r in rows[head + 1:]:
        if len(r) < len(cols) or r[cols["Metric Name"]] not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        if r[cols["Metric Unit"]] not in ("byte", "bytes"):
            raise ValueError(f"unexpected unit {r[cols['Metric Unit']]!r}: capture with --csv (base units)")
        L = launches.setdefault(int(r[cols["ID"]]), {"kernel": r[cols["Kernel Name"]]})
        L[r[cols["Metric Name"]]] = float(r[cols["Metric Value"]].replace(",", ""))
    seq = [launches[i] for i in sorted(launches)]
    names = [next(k for k in ("gates_kernel", "bp_kernel", "regauge_kernel") if k in L["kernel"]) for L in seq]
    if names != ["gates_kernel", "bp_kernel", "bp_kernel", "regauge_kernel"]:
        raise ValueError(f"expected the gates, two BP and the regauge launches, got {names}")
    tot = [L["dram__bytes_read.sum"] + L["dram__bytes_write.sum"] for L in seq]
    per_sweep = (tot[2] - tot[1]) / 20.0
    rec = {"mixed": {
        "chi": WL["chi"], "sources_sha256": sources_sha256(),
        "case": f"python bench.py --ncu-case {TRAFFIC_CASE} (n=1000, chi=4, mixed, 3-colour schedule, gates in "
                f"256-thread blocks; launches after layer {TRAFFIC_CASE})",
        "command": TRAFFIC_NCU,
        "gates_kernel": {"bytes_per_launch": tot[0]},
        "bp_kernel": {"fixed_bytes": tot[1] - per_sweep, "bytes_per_sweep": per_sweep,
                      "note": (f"1-sweep launch {seq[1]['dram__bytes_read.sum']:.0f} B read, "
                               f"{seq[1]['dram__bytes_write.sum']:.0f} B write; 21-sweep launch "
                               f"{seq[2]['dram__bytes_read.sum']:.0f} B read, {seq[2]['dram__bytes_write.sum']:.0f} B "
                               "write; per sweep = the difference / 20, fixed = the 1-sweep launch minus one sweep: "
                               "the sweeps run from L2")},
        "regauge_kernel": {"bytes_per_launch": tot[3]}}}
    with open(TRAFFIC_FILE, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    return rec


def main():
    a = parse()
    if a.traffic_record:
        print(json.dumps(traffic_record(a.traffic_record)))
        return
    if a.policy_study:
        policy_study(a)
        return
    if a.deg4_study:
        deg4_study(a)
        return
    if a.chi_sweep:
        chi_sweep(a)
        return
    if a.bp_study:
        bp_study(a)
        return
    if a.ncu_case is not None:
        ncu_case(a)
        return
    if a.ncu_scale is not None:
        ncu_scale(a)
        return
    if a.oracle_sample:
        print(json.dumps(oracle_sample_main(a.oracle_sample, a.budget)))
        return
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gtqa(a)


if __name__ == "__main__":
    main()
