"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and the
CPU oracle on the same seeded instance and compare gauge-invariant outputs."""
from __future__ import annotations

import numpy as np

from oracle import gtqa_oracle as O


def lib():
    from paper_2409_12240_gb300 import gtqa
    gtqa.load(build_if_missing=True)
    return gtqa


def oracle_padded_messages(st, msgs, chi_store):
    return O.messages_to_padded(st, msgs, chi_store)


def weighted_abs_gamma(G, L, inc_edges):
    """|Gamma_a| prod_k lambda_{e_k}[j_k] on the padded layout (phase-gauge invariant)."""
    n, _, C, _, _ = G.shape
    W = np.abs(G).copy()
    for a in range(n):
        for k in range(3):
            e = inc_edges[a][k] if k < len(inc_edges[a]) else -1
            lam = L[e] if e >= 0 else np.eye(C)[0]
            shape = [1, 1, 1, 1]
            shape[1 + k] = C
            W[a] *= lam.reshape(shape)
    return W


def message_spectra(M):
    Mh = 0.5 * (M + np.conj(np.swapaxes(M, -1, -2)))
    return np.linalg.eigvalsh(Mh)


def run_pair(inst, chi, K, dt, tol, max_iter, layers, precision=0, check_every=1, shape=None):
    """Run `layers` annealing layers on both sides; returns per-layer diffs.  `shape` (three
    variant indices) selects the launch shapes of the GPU side's phase kernels."""
    G = lib()
    opt = G.gtqa_options_init(precision=precision)
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour, opt)
    out = {"rho": [], "lam": [], "msg_abs": [], "msg_spec": [], "iters": [], "gamma": []}
    try:
        if shape is not None:
            G.gtqa_set_shape(s, shape)
            out["launch"] = G.gtqa_launch_shape(s)
        n, m, C, _ = G.gtqa_sizes(s)
        st = O.plus_state(inst.n, inst.edges)
        for k in range(1, layers + 1):
            G.gtqa_trotter_layer(s, k / K, dt)
            it_g, dist_g, _ = G.gtqa_bp_sweep(s, tol, max_iter)
            tZ, tX = O.schedule(k, K, dt)
            pre_dims = [l.size for l in st.lam]
            st, info = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, chi, tol, max_iter)
            out["iters"].append((it_g, info["bp_iters"]))
            if k % check_every and k != layers:
                continue
            rho_g, _ = G.gtqa_marginals(s)
            rho_o = O.reduced_density_matrices(st)
            out["rho"].append(float(np.abs(rho_g - rho_o).max()))
            Gg, Lg, Mg = G.gtqa_get_state(s)
            _, Lo = O.to_padded(st, C)
            out["lam"].append(float(np.abs(Lg - Lo).max()))
            Mo = np.zeros_like(Mg)
            for (e, d), mm in info["messages"].items():
                Mo[2 * e + d, :mm.shape[0], :mm.shape[1]] = mm
            out["msg_abs"].append(float(np.abs(np.abs(Mg) - np.abs(Mo)).max()))
            out["msg_spec"].append(float(np.abs(message_spectra(Mg) - message_spectra(Mo)).max()))
            Go, Lo2 = O.to_padded(st, C)
            Wg = weighted_abs_gamma(Gg, Lg, st.inc)
            Wo = weighted_abs_gamma(Go, Lo2, st.inc)
            out["gamma"].append(float(np.abs(Wg - Wo).max()))
        out["stats"] = G.gtqa_stats(s)
        out["state"] = st
        out["rho_gpu"] = G.gtqa_marginals(s)
    finally:
        G.gtqa_destroy(s)
    return out


def star_state(Gg, Lg, Mg, edges, inc, a):
    """The star of vertex a (a and its neighbours, a's edges in slot order) as an oracle state
    with a's Gamma and the messages into a; the neighbours' tensors are not used."""
    es = inc[a]
    nb = [int(edges[e][1] if edges[e][0] == a else edges[e][0]) for e in es]
    k = len(es)
    star_edges = np.array([[0, q + 1] for q in range(k)], dtype=np.int64)
    C = Gg.shape[2]
    Gs = np.zeros((k + 1,) + Gg.shape[1:], dtype=np.complex128)
    Gs[0] = Gg[a]
    Gs[1:, :, 0, 0, 0] = 1.0
    Ls = np.stack([Lg[e] for e in es])
    st = O.from_padded(k + 1, star_edges, Gs, Ls)
    msgs = {}
    for q, e in enumerate(es):
        d = st.lam[q].size
        inward = 2 * e + (0 if edges[e][0] == nb[q] else 1)    # m_{nb -> a}
        outward = 2 * e + (0 if edges[e][0] == a else 1)      # m_{a -> nb}
        msgs[(q, 1)] = np.array(Mg[inward, :d, :d])
        msgs[(q, 0)] = np.array(Mg[outward, :d, :d])
    return st, msgs
