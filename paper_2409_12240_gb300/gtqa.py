"""Python binding of the GTQA C ABI (include/gtqa.h).

Argument marshalling only: every step of the annealer runs in libgtqa.so.
Functions keep the C names.  Arrays may be numpy arrays (host) or CUDA torch
tensors (device; passed by data_ptr()).  There is no CPU fallback: if the
library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

from . import _build

GTQA_OK = 0
GTQA_ERR_INVALID_ARG = 1
GTQA_ERR_NOT_CONVERGED = 2
GTQA_ERR_NUMERIC = 3
GTQA_ERR_OOM = 4
GTQA_ERR_CUDA = 5
GTQA_ERR_TIMEOUT = 6
GTQA_ERR_UNSUPPORTED = 7

GTQA_FP64 = 0
GTQA_MIXED = 1
GTQA_C64 = 2

GTQA_BP_WARM_START = 1
GTQA_BP_REGAUGE = 2
GTQA_BP_DEFAULT = 3

GTQA_TROTTER_FIRST = 1
GTQA_TROTTER_SYMMETRIC = 2

EXPORTED = [
    "gtqa_options_init", "gtqa_create", "gtqa_create_batch", "gtqa_trotter_layer", "gtqa_bp_sweep",
    "gtqa_regauge", "gtqa_anneal", "gtqa_marginals", "gtqa_stats", "gtqa_get_state", "gtqa_set_state", "gtqa_sizes",
    "gtqa_edge_colouring", "gtqa_strerror", "gtqa_destroy", "gtqa_profile", "gtqa_profile_read",
    "gtqa_profile_name", "gtqa_alu_peak", "gtqa_debug_barrier", "gtqa_math_check", "gtqa_bp_static",
    "gtqa_barrier_bench", "gtqa_residual", "gtqa_entropy", "gtqa_spectral_bipartition", "gtqa_sample",
    "gtqa_trotter_split", "gtqa_anneal_ex", "gtqa_apply_gates", "gtqa_apply_single_qubit_gates",
    "gtqa_max_degree", "gtqa_anneal_graph", "gtqa_autotune", "gtqa_set_grid", "gtqa_gate_layers",
    "gtqa_anneal_policy", "gtqa_regauge_counts", "gtqa_set_shape", "gtqa_launch_shape",
]
KERNEL_KINDS = ["gates_kernel", "bp_kernel", "regauge_kernel", "marginals_kernel"]


class gtqa_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("svd_cutoff", ctypes.c_double), ("eig_cutoff", ctypes.c_double),
                ("cuda_stream", ctypes.c_void_p)]


class gtqa_stats_t(ctypes.Structure):
    _fields_ = [("layers", ctypes.c_int64), ("gates", ctypes.c_int64), ("last_bp_iters", ctypes.c_int32),
                ("not_converged", ctypes.c_int32), ("last_bp_dist", ctypes.c_double),
                ("discarded_weight", ctypes.c_double), ("log_fidelity", ctypes.c_double),
                ("svd_pairs", ctypes.c_int64), ("svd_rotations", ctypes.c_int64), ("bp_sweeps", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("bp_calls", ctypes.c_int64), ("bp_not_converged_calls", ctypes.c_int64),
                ("bp_exact_passes", ctypes.c_int64), ("regauge_svd_sweeps", ctypes.c_int64),
                ("gate_svd_sweeps_max", ctypes.c_int32), ("gate_svd_sweeps32_max", ctypes.c_int32),
                ("regauge_svd_sweeps_max", ctypes.c_int32), ("regauge_svd_sweeps32_max", ctypes.c_int32)]


class GTQAError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (code {code})")


_LIB: Optional[ctypes.CDLL] = None


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libgtqa.so (raises if it is missing and build_if_missing is False)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB_PATH
    if build_if_missing and _build.needs_build():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"GTQA CUDA library not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I32, I64, D, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint32
    sig = {
        "gtqa_options_init": (None, [ctypes.POINTER(gtqa_options)]),
        "gtqa_create": (I32, [I32, I32, P, P, P, P, I32, ctypes.POINTER(gtqa_options), ctypes.POINTER(P)]),
        "gtqa_create_batch": (I32, [I32, P, P, P, P, P, P, I32, ctypes.POINTER(gtqa_options), ctypes.POINTER(P)]),
        "gtqa_trotter_layer": (I32, [P, D, D]),
        "gtqa_bp_sweep": (I32, [P, D, I32, U32, ctypes.POINTER(I32), ctypes.POINTER(D)]),
        "gtqa_regauge": (I32, [P]),
        "gtqa_anneal": (I32, [P, I32, I32, I32, D, D, I32]),
        "gtqa_anneal_graph": (I32, [P, I32, I32, I32, D, D, I32]),
        "gtqa_anneal_policy": (I32, [P, I32, I32, I32, D, D, I32, D]),
        "gtqa_regauge_counts": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "gtqa_autotune": (I32, [P, D, D, D, I32, P]),
        "gtqa_set_grid": (I32, [P, P]),
        "gtqa_set_shape": (I32, [P, P]),
        "gtqa_launch_shape": (I32, [P, P]),
        "gtqa_gate_layers": (I32, [I32, I32, P, I32, P, P, ctypes.POINTER(I32)]),
        "gtqa_trotter_split": (I32, [P, D, D, D]),
        "gtqa_anneal_ex": (I32, [P, I32, I32, I32, D, D, I32, I32, P]),
        "gtqa_apply_gates": (I32, [P, I32, P, P]),
        "gtqa_apply_single_qubit_gates": (I32, [P, I32, P, P]),
        "gtqa_max_degree": (I32, [P, ctypes.POINTER(I32)]),
        "gtqa_marginals": (I32, [P, P, P]),
        "gtqa_residual": (I32, [P, ctypes.POINTER(D)]),
        "gtqa_entropy": (I32, [P, P, ctypes.POINTER(D)]),
        "gtqa_sample": (I32, [P, I32, P, P, D, I32, P, P]),
        "gtqa_spectral_bipartition": (I32, [I32, I32, P, P, P, ctypes.POINTER(D)]),
        "gtqa_stats": (I32, [P, ctypes.POINTER(gtqa_stats_t)]),
        "gtqa_get_state": (I32, [P, P, P, P]),
        "gtqa_set_state": (I32, [P, P, P, P]),
        "gtqa_sizes": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I32), ctypes.POINTER(I32)]),
        "gtqa_edge_colouring": (I32, [I32, I32, P, P, ctypes.POINTER(I32)]),
        "gtqa_strerror": (ctypes.c_char_p, [I32]),
        "gtqa_destroy": (None, [P]),
        "gtqa_profile": (I32, [P, I32]),
        "gtqa_profile_read": (I32, [P, I32, ctypes.POINTER(I64), ctypes.POINTER(D), ctypes.POINTER(I64)]),
        "gtqa_profile_name": (ctypes.c_char_p, [I32]),
        "gtqa_alu_peak": (I32, [I32, ctypes.POINTER(D)]),
        "gtqa_debug_barrier": (I32, [P, I64, I32]),
        "gtqa_math_check": (I32, [I32, P, P]),
        "gtqa_barrier_bench": (I32, [I32, I32, ctypes.POINTER(D)]),
        "gtqa_bp_static": (I32, [I32, I32, P, P, P, P, P, D, I32, ctypes.POINTER(I32), ctypes.POINTER(D), P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def strerror(code: int) -> str:
    return load().gtqa_strerror(int(code)).decode()


def _ptr(a) -> Tuple[int, object]:
    """(address, keep-alive) of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return 0, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_contiguous"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return int(a.data_ptr()), a
    if not (a.flags["C_CONTIGUOUS"]):
        raise ValueError("array must be C-contiguous")
    return int(a.ctypes.data), a


def _check(code: int, where: str, allow=(GTQA_OK,)) -> int:
    if code not in allow:
        raise GTQAError(code, where)
    return code


def gtqa_options_init(precision: int = GTQA_FP64, svd_cutoff: float = 0.0, eig_cutoff: float = 0.0,
                      cuda_stream: int = 0) -> gtqa_options:
    o = gtqa_options()
    load().gtqa_options_init(ctypes.byref(o))
    o.precision = precision
    if svd_cutoff > 0:
        o.svd_cutoff = svd_cutoff
    if eig_cutoff > 0:
        o.eig_cutoff = eig_cutoff
    o.cuda_stream = cuda_stream or None
    return o


def gtqa_create(n: int, edges, J, h, chi: int, colour=None, opt: Optional[gtqa_options] = None) -> int:
    """Create a single-instance state; returns the opaque handle (an int)."""
    edges = np.ascontiguousarray(edges, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    col = None if colour is None else np.ascontiguousarray(colour, dtype=np.int32)
    handle = ctypes.c_void_p()
    m = int(edges.shape[0]) if edges.size else 0
    rc = load().gtqa_create(int(n), m, _ptr(edges)[0] or None, _ptr(col)[0] or None, _ptr(J)[0] or None,
                            _ptr(h)[0], int(chi), ctypes.byref(opt) if opt is not None else None,
                            ctypes.byref(handle))
    _check(rc, "gtqa_create")
    return int(handle.value)


def gtqa_create_batch(ns: Sequence[int], edges_list, J_list, h_list, chi: int, colour_list=None,
                      opt: Optional[gtqa_options] = None) -> int:
    """Create B instances evolving together; arrays are given per instance."""
    B = len(ns)
    n = np.ascontiguousarray(ns, dtype=np.int32)
    m = np.ascontiguousarray([len(e) for e in edges_list], dtype=np.int32)
    edges = np.ascontiguousarray(np.concatenate([np.asarray(e, dtype=np.int32).reshape(-1, 2) for e in edges_list]))
    J = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64) for x in J_list]))
    h = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64) for x in h_list]))
    col = None
    if colour_list is not None:
        col = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.int32) for c in colour_list]))
    handle = ctypes.c_void_p()
    rc = load().gtqa_create_batch(B, _ptr(n)[0], _ptr(m)[0], _ptr(edges)[0], _ptr(col)[0] or None, _ptr(J)[0],
                                  _ptr(h)[0], int(chi), ctypes.byref(opt) if opt is not None else None,
                                  ctypes.byref(handle))
    _check(rc, "gtqa_create_batch")
    return int(handle.value)


def gtqa_trotter_layer(s: int, tau: float, dt: float) -> None:
    _check(load().gtqa_trotter_layer(s, float(tau), float(dt)), "gtqa_trotter_layer")


def gtqa_bp_sweep(s: int, tol: float, max_iter: int, flags: int = GTQA_BP_DEFAULT,
                  raise_not_converged: bool = False) -> Tuple[int, float, bool]:
    """Returns (sweeps run, final dist/|E|, converged)."""
    it = ctypes.c_int32()
    d = ctypes.c_double()
    allow = (GTQA_OK,) if raise_not_converged else (GTQA_OK, GTQA_ERR_NOT_CONVERGED)
    rc = _check(load().gtqa_bp_sweep(s, float(tol), int(max_iter), int(flags), ctypes.byref(it), ctypes.byref(d)),
                "gtqa_bp_sweep", allow)
    return int(it.value), float(d.value), rc == GTQA_OK


def gtqa_regauge(s: int) -> None:
    _check(load().gtqa_regauge(s), "gtqa_regauge")


def gtqa_anneal(s: int, k_begin: int, k_end: int, K: int, dt: float, tol: float, max_iter: int) -> None:
    """Layers k_begin..k_end of the K-layer anneal in one persistent launch (asynchronous)."""
    _check(load().gtqa_anneal(s, int(k_begin), int(k_end), int(K), float(dt), float(tol), int(max_iter)),
           "gtqa_anneal")


def gtqa_trotter_split(s: int, t_Z: float, t_X_pre: float, t_X_post: float) -> None:
    """One layer U_X(t_X_post) U_Z(t_Z) U_X(t_X_pre) (asynchronous)."""
    _check(load().gtqa_trotter_split(s, float(t_Z), float(t_X_pre), float(t_X_post)), "gtqa_trotter_split")


def gtqa_anneal_ex(s: int, k_begin: int, k_end: int, K: int, dt: float, tol: float, max_iter: int,
                   order: int = GTQA_TROTTER_FIRST, reverse=None) -> None:
    """gtqa_anneal with the first-order (optionally reversed per layer) or symmetric formula."""
    rv = None if reverse is None else np.ascontiguousarray(np.asarray(reverse, dtype=np.uint8))
    if rv is not None and rv.size != k_end - k_begin + 1:
        raise ValueError("reverse needs one entry per layer")
    _check(load().gtqa_anneal_ex(s, int(k_begin), int(k_end), int(K), float(dt), float(tol), int(max_iter),
                                 int(order), rv.ctypes.data if rv is not None else None), "gtqa_anneal_ex")


def gtqa_apply_gates(s: int, edge, U) -> None:
    """Arbitrary two-qubit gates, U[q] a 4x4 complex matrix on edge[q] (asynchronous)."""
    e = np.ascontiguousarray(np.asarray(edge, dtype=np.int32).reshape(-1))
    u = np.ascontiguousarray(np.asarray(U, dtype=np.complex128).reshape(-1, 4, 4))
    if u.shape[0] != e.size:
        raise ValueError("one 4x4 matrix per gate")
    _check(load().gtqa_apply_gates(s, int(e.size), e.ctypes.data if e.size else None,
                                   u.ctypes.data if e.size else None), "gtqa_apply_gates")


def gtqa_apply_single_qubit_gates(s: int, vertex, W) -> None:
    """Arbitrary one-qubit gates, W[q] a 2x2 complex matrix on vertex[q] (asynchronous)."""
    v = np.ascontiguousarray(np.asarray(vertex, dtype=np.int32).reshape(-1))
    w = np.ascontiguousarray(np.asarray(W, dtype=np.complex128).reshape(-1, 2, 2))
    if w.shape[0] != v.size:
        raise ValueError("one 2x2 matrix per gate")
    _check(load().gtqa_apply_single_qubit_gates(s, int(v.size), v.ctypes.data if v.size else None,
                                                w.ctypes.data if v.size else None), "gtqa_apply_single_qubit_gates")


def gtqa_anneal_graph(s: int, k_begin: int, k_end: int, K: int, dt: float, tol: float, max_iter: int) -> None:
    """gtqa_anneal replayed from a CUDA graph captured once per argument set (asynchronous)."""
    _check(load().gtqa_anneal_graph(s, int(k_begin), int(k_end), int(K), float(dt), float(tol), int(max_iter)),
           "gtqa_anneal_graph")


def gtqa_autotune(s: int, tau: float, dt: float, tol: float, max_iter: int) -> Tuple[int, int, int]:
    """Time each phase kernel's launch-shape variants and candidate grid sizes on the current
    state; keep the fastest and return the grid sizes (gates, BP, regauge)."""
    g = np.zeros(3, dtype=np.int32)
    _check(load().gtqa_autotune(s, float(tau), float(dt), float(tol), int(max_iter), g.ctypes.data), "gtqa_autotune")
    return int(g[0]), int(g[1]), int(g[2])


def gtqa_set_grid(s: int, grid) -> None:
    g = np.ascontiguousarray(np.asarray(grid, dtype=np.int32))
    _check(load().gtqa_set_grid(s, g.ctypes.data), "gtqa_set_grid")


def gtqa_set_shape(s: int, variant) -> None:
    """Launch-shape variant per phase kernel (gates 0-1, BP 0-2, regauge 0-2)."""
    v = np.ascontiguousarray(np.asarray(variant, dtype=np.int32))
    if v.shape != (3,):
        raise ValueError("gtqa_set_shape: three variants (gates, BP, regauge)")
    _check(load().gtqa_set_shape(s, v.ctypes.data), "gtqa_set_shape")


def gtqa_launch_shape(s: int) -> dict:
    """The launch table: per kernel its grid, variant, threads per block and team size."""
    out = np.zeros(12, dtype=np.int32)
    _check(load().gtqa_launch_shape(s, out.ctypes.data), "gtqa_launch_shape")
    return {k: {"grid": int(out[4 * q]), "variant": int(out[4 * q + 1]), "threads_per_block": int(out[4 * q + 2]),
                "team": int(out[4 * q + 3])} for q, k in enumerate(KERNEL_KINDS[:3])}


def gtqa_gate_layers(n: int, edges, edge) -> Tuple[np.ndarray, int]:
    """Host-only: (launch of each gate, number of launches) of gtqa_apply_gates' layering."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    g = np.ascontiguousarray(np.asarray(edge, dtype=np.int32).reshape(-1))
    lay = np.zeros(max(g.size, 1), dtype=np.int32)
    nl = ctypes.c_int32()
    _check(load().gtqa_gate_layers(int(n), int(e.shape[0]), e.ctypes.data, int(g.size), g.ctypes.data, lay.ctypes.data,
                                   ctypes.byref(nl)), "gtqa_gate_layers")
    return lay[:g.size], int(nl.value)


def gtqa_anneal_policy(s: int, k_begin: int, k_end: int, K: int, dt: float, tol: float, max_iter: int,
                       r_threshold: float) -> None:
    """gtqa_anneal, regauging only the layers whose residual R exceeds r_threshold."""
    _check(load().gtqa_anneal_policy(s, int(k_begin), int(k_end), int(K), float(dt), float(tol), int(max_iter),
                                     float(r_threshold)), "gtqa_anneal_policy")


def gtqa_regauge_counts(s: int) -> Tuple[int, int]:
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().gtqa_regauge_counts(s, ctypes.byref(a), ctypes.byref(b)), "gtqa_regauge_counts")
    return int(a.value), int(b.value)


def gtqa_sizes(s: int) -> Tuple[int, int, int, int]:
    n, m, c, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().gtqa_sizes(s, ctypes.byref(n), ctypes.byref(m), ctypes.byref(c), ctypes.byref(k)), "gtqa_sizes")
    return int(n.value), int(m.value), int(c.value), int(k.value)


def gtqa_sample(s: int, order, u, tol: float, max_iter: int) -> Tuple[np.ndarray, np.ndarray]:
    """BP-guided measurement sampling (Sec. IV A); returns (x, p)."""
    o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    n = gtqa_sizes(s)[0]
    x = np.zeros(n, dtype=np.int8)
    p = np.zeros(max(o.size, 1), dtype=np.float64)
    _check(load().gtqa_sample(s, int(o.size), o.ctypes.data, uu.ctypes.data, float(tol), int(max_iter), x.ctypes.data,
                              p.ctypes.data), "gtqa_sample")
    return x, p[:o.size]


def gtqa_entropy(s: int, cut) -> float:
    """Mean-field entanglement entropy of the bipartition whose cut edges are marked in `cut`
    (Sec. III C, Eq. (apprx_entropy))."""
    c = np.ascontiguousarray(np.asarray(cut).astype(np.uint8))
    v = ctypes.c_double()
    _check(load().gtqa_entropy(s, c.ctypes.data, ctypes.byref(v)), "gtqa_entropy")
    return float(v.value)


def gtqa_spectral_bipartition(n: int, edges) -> Tuple[np.ndarray, np.ndarray, float]:
    """Eq. (bipartition) by spectral partitioning: returns (side, cut, ratio)."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    side = np.zeros(int(n), dtype=np.uint8)
    cut = np.zeros(e.shape[0], dtype=np.uint8)
    r = ctypes.c_double()
    _check(load().gtqa_spectral_bipartition(int(n), int(e.shape[0]), e.ctypes.data, side.ctypes.data,
                                            cut.ctypes.data, ctypes.byref(r)), "gtqa_spectral_bipartition")
    return side.astype(bool), cut.astype(bool), float(r.value)


def gtqa_residual(s: int) -> float:
    """Local-orthogonality residual R of the current state (App. C)."""
    r = ctypes.c_double()
    _check(load().gtqa_residual(s, ctypes.byref(r)), "gtqa_residual")
    return float(r.value)


def gtqa_marginals(s: int, rho_out=None, sign_out=None):
    """rho (n, 2, 2) complex128 and signs (n,) int8.  Allocates host arrays if none given."""
    n, _, _, _ = gtqa_sizes(s)
    if rho_out is None:
        rho_out = np.zeros((n, 2, 2), dtype=np.complex128)
    if sign_out is None:
        sign_out = np.zeros(n, dtype=np.int8)
    _check(load().gtqa_marginals(s, _ptr(rho_out)[0], _ptr(sign_out)[0] or None), "gtqa_marginals")
    return rho_out, sign_out


def gtqa_stats(s: int) -> dict:
    st = gtqa_stats_t()
    _check(load().gtqa_stats(s, ctypes.byref(st)), "gtqa_stats")
    return {k: getattr(st, k) for k, _ in gtqa_stats_t._fields_}


def gtqa_max_degree(s: int) -> int:
    D = ctypes.c_int32()
    _check(load().gtqa_max_degree(s, ctypes.byref(D)), "gtqa_max_degree")
    return int(D.value)


def gtqa_get_state(s: int):
    """(Gamma (n,2,CHI,...,CHI) complex128 with one CHI per bond slot, lambda (m,CHI),
    messages (2m,CHI,CHI) complex128)."""
    n, m, C, _ = gtqa_sizes(s)
    G = np.zeros((n, 2) + (C,) * gtqa_max_degree(s), dtype=np.complex128)
    L = np.zeros((m, C), dtype=np.float64)
    Mg = np.zeros((2 * m, C, C), dtype=np.complex128)
    _check(load().gtqa_get_state(s, _ptr(G)[0], _ptr(L)[0], _ptr(Mg)[0]), "gtqa_get_state")
    return G, L, Mg


def gtqa_set_state(s: int, G, L, Mg) -> None:
    G = np.ascontiguousarray(G, dtype=np.complex128)
    L = np.ascontiguousarray(L, dtype=np.float64)
    Mg = np.ascontiguousarray(Mg, dtype=np.complex128)
    _check(load().gtqa_set_state(s, _ptr(G)[0], _ptr(L)[0], _ptr(Mg)[0]), "gtqa_set_state")


def gtqa_edge_colouring(n: int, edges) -> Tuple[np.ndarray, int]:
    edges = np.ascontiguousarray(edges, dtype=np.int32)
    col = np.zeros(edges.shape[0], dtype=np.int32)
    k = ctypes.c_int32()
    _check(load().gtqa_edge_colouring(int(n), int(edges.shape[0]), _ptr(edges)[0], _ptr(col)[0], ctypes.byref(k)),
           "gtqa_edge_colouring")
    return col, int(k.value)


def gtqa_profile(s: int, enable: bool) -> None:
    _check(load().gtqa_profile(s, 1 if enable else 0), "gtqa_profile")


def gtqa_profile_read(s: int) -> dict:
    """{kernel class: (launches, total ms, units)} for every class."""
    out = {}
    for k, name in enumerate(KERNEL_KINDS):
        l, ms, u = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
        _check(load().gtqa_profile_read(s, k, ctypes.byref(l), ctypes.byref(ms), ctypes.byref(u)), "gtqa_profile_read")
        out[name] = (int(l.value), float(ms.value), int(u.value))
    return out


def gtqa_profile_name(kind: int) -> Optional[str]:
    r = load().gtqa_profile_name(int(kind))
    return None if r is None else r.decode()


def gtqa_alu_peak(fp64: bool) -> float:
    """Measured FMA throughput (TFLOP/s) of the current device."""
    t = ctypes.c_double()
    _check(load().gtqa_alu_peak(1 if fp64 else 0, ctypes.byref(t)), "gtqa_alu_peak")
    return float(t.value)


def gtqa_debug_barrier(s: int, spin_limit: int, extra_arrivals: int) -> None:
    _check(load().gtqa_debug_barrier(s, int(spin_limit), int(extra_arrivals)), "gtqa_debug_barrier")


def gtqa_math_check(x) -> np.ndarray:
    """(n, 6): refined 1/x, CUDA 1/x, refined x^-1/2, CUDA x^-1/2, refined sqrt, CUDA sqrt."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros((x.size, 6))
    _check(load().gtqa_math_check(int(x.size), _ptr(x)[0], _ptr(out)[0]), "gtqa_math_check")
    return out


def gtqa_bp_static(n: int, m: int, vert_edges, edge_info, gamma, lam, messages_out, tol: float,
                   max_iter: int, cuda_stream: int = 0) -> Tuple[int, int, float]:
    """BP without device allocation on caller-owned device buffers (torch CUDA tensors).
    Returns (status code, sweeps run, final dist/|E|); raises on errors other than
    GTQA_ERR_NOT_CONVERGED."""
    it = ctypes.c_int32()
    d = ctypes.c_double()
    rc = load().gtqa_bp_static(int(n), int(m), _ptr(vert_edges)[0], _ptr(edge_info)[0], _ptr(gamma)[0],
                               _ptr(lam)[0], _ptr(messages_out)[0], float(tol), int(max_iter), ctypes.byref(it),
                               ctypes.byref(d), cuda_stream or None)
    _check(rc, "gtqa_bp_static", (GTQA_OK, GTQA_ERR_NOT_CONVERGED))
    return rc, int(it.value), float(d.value)


def gtqa_barrier_bench(threads: int = 512, rounds: int = 2000) -> float:
    """Microseconds per grid barrier (cooperative launch, one block per SM)."""
    us = ctypes.c_double()
    _check(load().gtqa_barrier_bench(int(threads), int(rounds), ctypes.byref(us)), "gtqa_barrier_bench")
    return float(us.value)


def gtqa_destroy(s: int) -> None:
    if s:
        load().gtqa_destroy(s)


class Annealer:
    """Convenience owner of one state handle: layer(), marginals(), close()."""

    def __init__(self, n, edges, J, h, chi, colour=None, precision=GTQA_FP64, cuda_stream=0, batch=None):
        opt = gtqa_options_init(precision=precision, cuda_stream=cuda_stream)
        if batch is None:
            self.handle = gtqa_create(n, edges, J, h, chi, colour, opt)
        else:
            ns, el, Jl, hl, cl = batch
            self.handle = gtqa_create_batch(ns, el, Jl, hl, chi, cl, opt)

    def layer(self, tau: float, dt: float, tol: float, max_iter: int) -> Tuple[int, float, bool]:
        gtqa_trotter_layer(self.handle, tau, dt)
        return gtqa_bp_sweep(self.handle, tol, max_iter, GTQA_BP_DEFAULT)

    def marginals(self):
        return gtqa_marginals(self.handle)

    def close(self):
        gtqa_destroy(self.handle)
        self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
