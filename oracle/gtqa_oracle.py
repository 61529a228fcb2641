"""Plain complex128 CPU oracle of the graph tensor-network quantum annealer (GTQA).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct restatement
of arXiv:2409.12240 used to check the CUDA path.  Only the test-suite, the
package's smoke check and the benchmark's CPU-baseline leg may import it; the
library itself never calls into it and shares no code with it.

Every step follows the paper's notation and order:

* graph tensor network and Vidal gauge ........ Sec. II A-C, Eq. (graph_tn), Eq. (vidal_gauge_tn)
* single-qubit gate in the Vidal gauge ........ Sec. II D
* two-qubit gate (simple update) .............. App. E (dense Theta SVD)
* truncation .................................. App. D, Algorithm "Truncation"
* symmetric split + warm-start messages ....... Sec. II C, Eq. (symmetric_gauge), Eq. (reconstructed_messages)
* belief propagation .......................... App. B, Algorithm "Belief propagation"; Eq. (local_consistency)
* Vidal gauge from messages (regauge) ......... App. D, Algorithm "Vidal gauge finding"
* local-orthogonality residual R .............. App. C
* reduced density matrices and read-out ....... Eq. (partial_dens), Eq. (bp_approx), Eq. (rounding_rule)
* Trotterised annealing schedule .............. App. F, Eq. (discretizatoion)
* per-gate fidelity estimate .................. Sec. III D, Eq. (gate_fidelity)
* mean-field entanglement entropy, bipartition . Sec. III C, Eqs. (bipartition), (mean_field_schmidt), (apprx_entropy)
* measurement sampling ........................ Sec. IV A, Eq. (projection)
* regauge only when R is large ................ Sec. II C, App. C (reading R15)
* other product formulas, arbitrary gates ..... Sec. V (second-order and randomised formulas);
                                                Sec. II D and App. E (any one- and two-qubit gate)

Readings taken where the paper is silent or ambiguous (each one is listed in the
design notes of the repository):

R1  Trotter order: layer k = 1..K is applied in time order; inside a layer the
    interaction layer U_Z acts first, then the mixing layer U_X.  The schedule
    s(t) = 1 - t/T is sampled at t = k dt, so with tau_k = k/K the Ising angle is
    t_Z = dt*tau_k and the mixing angle is t_X = dt*(1 - tau_k).
R2  Gate order inside U_Z: colour classes of a proper edge colouring in
    ascending colour, edges of one colour in ascending edge id (gates of one
    colour commute).
R3  Warm start: m_{a->b} = diag(lambda_ab)/sum(lambda_ab).  The printed formula
    uses lambda^{1/2}; with T = Gamma lambda^{1/2} the local-orthogonality
    condition makes diag(lambda) the fixed point.  `paper_sqrt_warmstart=True`
    reproduces the printed formula.
R4  BP schedule: flooding (all messages of a sweep computed from the previous
    sweep).  The printed algorithm replaces messages inside the edge loop; that
    sequential schedule is available as schedule="sequential".
R5  Distance: dist = sum over the 2|E| directed messages of the trace norm
    (sum of singular values) of new - old; stop when dist/|E| < tol, at most
    max_iter sweeps.
R6  Cut-offs: singular values s <= svd_cutoff * s_0 are dropped (the bond
    shrinks); message eigenvalues w <= eig_cutoff * w_max are treated as zero in
    both m^{1/2} and m^{-1/2} (pseudo-inverse).  Messages are made exactly
    Hermitian, (m + m^H)/2, before their eigen-decomposition.
R7  Normalisation: after every SVD the kept singular values are normalised to
    unit 2-norm.  In the regauge the two bond transforms are each scaled by
    ||S||^{1/2}, so that the represented state is unchanged while lambda is
    normalised (the printed algorithm leaves ||S|| in lambda).
R8  Marginals: Eq. (partial_dens) with the environment of Eq. (bp_approx) built
    from the warm-start messages of the current Vidal-gauge state, i.e.
    rho_a = sum Gamma Gamma^* prod_b lambda_ba^2, divided by its trace.
R9  Read-out tie rho_a[0,0] = 1/2 maps to -1 (literal "otherwise").
R13 Product formulas beyond first order (the paper names them only as an
    outlook, Sec. V): a layer is U_X(t_post) U_Z(t_Z) U_X(t_pre).  First order
    (R1) is (t_pre, t_post) = (0, t_X); the second-order symmetric (Strang)
    formula is (t_X/2, t_X/2) at the same tau_k; the randomised first-order
    formula draws, per layer, the forward (0, t_X) or the reversed (t_X, 0)
    ordering with probability 1/2 each (the caller supplies the draws).
R15 Regauge policy (Sec. II C: the paper regauges occasionally, when R grows too
    large): after the Trotter layer, R of App. C is evaluated, and the symmetric
    split, BP and Vidal gauge finding run only if R > r_threshold.  A negative
    threshold regauges every layer (R1-R14).
R14 Arbitrary two-qubit gate on edge e = {a, b} with a = edges[e][0]: a 4x4
    matrix W[(i_a i_b), (i_a' i_b')] (row index 2 i_a + i_b), applied by the
    same simple update as the Ising gate (App. E); gates are applied in the
    order given.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

SVD_CUTOFF = 1e-14
EIG_CUTOFF = 1e-13


# --------------------------------------------------------------------------
# graph bookkeeping
# --------------------------------------------------------------------------
@dataclasses.dataclass
class VidalState:
    """Graph tensor network in the Vidal gauge, Eq. (vidal_gauge_tn).

    Gamma[a] has shape (2, d_{e_0}, ..., d_{e_{k-1}}) where e_0 < ... < e_{k-1} are
    the edges incident to a (its bond "slots", ascending edge id).  lam[e] is the
    vector lambda_e of length d_e.
    """
    n: int
    edges: np.ndarray                 # (m, 2), u < v
    inc: List[List[int]]              # incident edge ids per vertex, ascending
    Gamma: List[np.ndarray]
    lam: List[np.ndarray]

    @property
    def m(self) -> int:
        return int(self.edges.shape[0])

    def slot(self, a: int, e: int) -> int:
        return self.inc[a].index(e)

    def other(self, e: int, a: int) -> int:
        u, v = self.edges[e]
        return int(v) if a == u else int(u)

    def copy(self) -> "VidalState":
        return VidalState(self.n, self.edges.copy(), [list(x) for x in self.inc],
                          [g.copy() for g in self.Gamma], [l.copy() for l in self.lam])


def incidence(n: int, edges: np.ndarray) -> List[List[int]]:
    inc: List[List[int]] = [[] for _ in range(n)]
    for e, (u, v) in enumerate(np.asarray(edges).tolist()):
        inc[u].append(e)
        inc[v].append(e)
    return inc


def plus_state(n: int, edges: np.ndarray) -> VidalState:
    """|+>^N as a Vidal-gauge network with all bond dimensions 1 (Sec. III A)."""
    edges = np.asarray(edges, dtype=np.int64)
    inc = incidence(n, edges)
    Gamma = []
    for a in range(n):
        g = np.zeros((2,) + (1,) * len(inc[a]), dtype=np.complex128)
        g[(0,) + (0,) * len(inc[a])] = 1 / np.sqrt(2)
        g[(1,) + (0,) * len(inc[a])] = 1 / np.sqrt(2)
        Gamma.append(g)
    lam = [np.ones(1) for _ in range(edges.shape[0])]
    return VidalState(n, edges, inc, Gamma, lam)


def directed(st: VidalState, a: int, e: int) -> Tuple[int, int]:
    """Key of message m_{a->b} for edge e = {a, b}: (e, 0) if a is edges[e][0], else (e, 1)."""
    return (e, 0) if int(st.edges[e][0]) == a else (e, 1)


def _scale_slot(t: np.ndarray, slot: int, vec: np.ndarray) -> np.ndarray:
    shape = [1] * t.ndim
    shape[1 + slot] = vec.size
    return t * vec.reshape(shape)


# --------------------------------------------------------------------------
# gates (App. F)
# --------------------------------------------------------------------------
def schedule(k: int, K: int, dt: float) -> Tuple[float, float]:
    """Angles of Trotter layer k (1-based), reading R1 of Eq. (discretizatoion).

    Returns (t_Z, t_X) = (dt * k/K, dt * (1 - k/K)).
    """
    tau = k / K
    return dt * tau, dt * (1.0 - tau)


def ising_gate(J: float, h_a: float, h_b: float, D_a: int, D_b: int, t: float) -> np.ndarray:
    """Two-qubit factor of U_Z(t) (App. F): exp(-i t (J Z_a Z_b + h_a/D_a Z_a + h_b/D_b Z_b)).

    Returned as a rank-4 tensor W[i_a, i_b, i_a', i_b'] (diagonal), with the Pauli
    eigenvalue z = +1 for |0> and -1 for |1>.
    """
    W = np.zeros((2, 2, 2, 2), dtype=np.complex128)
    for ia in range(2):
        for ib in range(2):
            za, zb = 1 - 2 * ia, 1 - 2 * ib
            W[ia, ib, ia, ib] = np.exp(-1j * t * (J * za * zb + h_a / D_a * za + h_b / D_b * zb))
    return W


def mixing_gate(t: float) -> np.ndarray:
    """Single-qubit factor of U_X(t) (App. F): exp(-i t X) = cos t I - i sin t X."""
    c, s = np.cos(t), np.sin(t)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def apply_single_qubit_gate(st: VidalState, a: int, W: np.ndarray) -> None:
    """Sec. II D: Gamma~_a[i, j] = sum_i' W[i, i'] Gamma_a[i', j]."""
    st.Gamma[a] = np.tensordot(W, st.Gamma[a], axes=([1], [0]))


# --------------------------------------------------------------------------
# simple update and truncation (App. E, App. D Algorithm "Truncation")
# --------------------------------------------------------------------------
def truncate(st: VidalState, e: int, chi_new: int) -> None:
    """Algorithm "Truncation": keep the first chi_new entries of lambda_e and slice
    Gamma_a, Gamma_b on that bond (lambda must be sorted descending)."""
    st.lam[e] = st.lam[e][:chi_new].copy()
    for x in (int(st.edges[e][0]), int(st.edges[e][1])):
        s = st.slot(x, e)
        idx = [slice(None)] * st.Gamma[x].ndim
        idx[1 + s] = slice(0, chi_new)
        st.Gamma[x] = st.Gamma[x][tuple(idx)].copy()


def simple_update(st: VidalState, e: int, W: np.ndarray, chi: int,
                  svd_cutoff: float = SVD_CUTOFF) -> Dict[str, float]:
    """Apply the two-qubit gate W to edge e = {a, b} (App. E) and truncate to chi.

    Theta[i_a, J_a, i_b, J_b] = sum W[i_a,i_b,i_a',i_b'] Gamma_a[i_a',J_a,j] Gamma_b[i_b',J_b,j]
                                 lambda_ab[j] prod lambda_ca prod lambda_cb,
    U, lambda, V^H = SVD(Theta), Gamma~_a = U / prod lambda_ca, Gamma~_b = V^* / prod lambda_cb.
    Singular values <= svd_cutoff * s_0 are dropped, at most chi are kept
    (Algorithm "Truncation"), and the kept ones are normalised (reading R7).

    Returns the discarded weight w = sum_{dropped} s^2 / sum s^2 and the gate
    fidelity estimate f = (1 - w)^2 of Eq. (gate_fidelity).
    """
    a, b = int(st.edges[e][0]), int(st.edges[e][1])
    sa, sb = st.slot(a, e), st.slot(b, e)

    def branch(x: int, s: int) -> Tuple[np.ndarray, Tuple[int, ...], np.ndarray]:
        X = st.Gamma[x]
        others = [k for k in range(len(st.inc[x])) if k != s]
        wgt = np.ones(1)
        for k in others:
            X = _scale_slot(X, k, st.lam[st.inc[x][k]])
        X = np.moveaxis(X, 1 + s, -1)                 # (2, J..., d_ab)
        other_dims = X.shape[1:-1]
        # prod of the neighbouring lambda's over the flattened J index
        wgt = np.ones(other_dims, dtype=np.float64)
        for pos, k in enumerate(others):
            shape = [1] * len(other_dims)
            shape[pos] = st.lam[st.inc[x][k]].size
            wgt = wgt * st.lam[st.inc[x][k]].reshape(shape)
        return X.reshape(2, -1, X.shape[-1]), other_dims, wgt.reshape(-1)

    Xa, dims_a, wa = branch(a, sa)
    Xb, dims_b, wb = branch(b, sb)
    lab = st.lam[e]
    Theta = np.einsum("xyab,apj,bqj,j->xpyq", W, Xa, Xb, lab)
    P, Q = Theta.shape[0] * Theta.shape[1], Theta.shape[2] * Theta.shape[3]
    U, s, Vh = np.linalg.svd(Theta.reshape(P, Q), full_matrices=False)
    total = float(np.sum(s ** 2))
    keep = int(np.sum(s > svd_cutoff * s[0])) if s[0] > 0 else 0
    keep = max(1, min(chi, keep))
    w = float(np.sum(s[keep:] ** 2) / total) if total > 0 else 0.0
    lam_new = s[:keep] / np.linalg.norm(s[:keep])
    inv_a = np.where(wa > 0, 1.0 / np.where(wa > 0, wa, 1.0), 0.0)
    inv_b = np.where(wb > 0, 1.0 / np.where(wb > 0, wb, 1.0), 0.0)
    Ga = U[:, :keep].reshape(2, -1, keep) * inv_a[None, :, None]
    Gb = Vh[:keep, :].T.reshape(2, -1, keep) * inv_b[None, :, None]
    Ga = np.moveaxis(Ga.reshape((2,) + tuple(dims_a) + (keep,)), -1, 1 + sa)
    Gb = np.moveaxis(Gb.reshape((2,) + tuple(dims_b) + (keep,)), -1, 1 + sb)
    st.Gamma[a], st.Gamma[b], st.lam[e] = Ga, Gb, lam_new
    return {"discarded": w, "fidelity": (1.0 - w) ** 2}


def trotter_layer(st: VidalState, colour: np.ndarray, J: np.ndarray, h: np.ndarray,
                  t_Z: float, t_X: float, chi: int, svd_cutoff: float = SVD_CUTOFF,
                  t_X_pre: float = 0.0) -> Dict[str, float]:
    """U_X(t_X) U_Z(t_Z) U_X(t_X_pre) of Eq. (discretizatoion) and reading R13: the
    leading mixing gate on every qubit (skipped for t_X_pre = 0), every edge gate of
    the interaction layer (colour classes ascending, reading R2), then the mixing
    gate on every qubit."""
    if t_X_pre != 0.0:
        Wp = mixing_gate(t_X_pre)
        for a in range(st.n):
            apply_single_qubit_gate(st, a, Wp)
    deg = [len(x) for x in st.inc]
    order = sorted(range(st.m), key=lambda e: (int(colour[e]), e))
    disc, logf = 0.0, 0.0
    for e in order:
        a, b = int(st.edges[e][0]), int(st.edges[e][1])
        W = ising_gate(float(J[e]), float(h[a]), float(h[b]), deg[a], deg[b], t_Z)
        r = simple_update(st, e, W, chi, svd_cutoff)
        disc += r["discarded"]
        logf += np.log(r["fidelity"]) if r["fidelity"] > 0 else -np.inf
    Wx = mixing_gate(t_X)
    for a in range(st.n):
        apply_single_qubit_gate(st, a, Wx)
    return {"discarded": disc, "log_fidelity": logf}


# --------------------------------------------------------------------------
# belief propagation (Sec. II B-C, App. A-B)
# --------------------------------------------------------------------------
def symmetric_gauge_vertex(st: VidalState, a: int) -> np.ndarray:
    """Eq. (symmetric_gauge) for one vertex: T_a = Gamma_a prod_b lambda_ba^{1/2}."""
    t = st.Gamma[a]
    for k, e in enumerate(st.inc[a]):
        t = _scale_slot(t, k, np.sqrt(st.lam[e]))
    return t


def symmetric_gauge(st: VidalState) -> List[np.ndarray]:
    """Eq. (symmetric_gauge) for every vertex."""
    return [symmetric_gauge_vertex(st, a) for a in range(st.n)]


def reconstructed_messages(st: VidalState, paper_sqrt_warmstart: bool = False) -> Dict[Tuple[int, int], np.ndarray]:
    """Warm-start messages of Eq. (reconstructed_messages), reading R3:
    m_{a->b} = diag(lambda_ab) / sum lambda_ab (both directions)."""
    msgs = {}
    for e in range(st.m):
        lam = np.sqrt(st.lam[e]) if paper_sqrt_warmstart else st.lam[e]
        m = np.diag(lam / lam.sum()).astype(np.complex128)
        msgs[(e, 0)] = m
        msgs[(e, 1)] = m.copy()
    return msgs


def random_messages(st: VidalState, A: Dict[Tuple[int, int], np.ndarray]) -> Dict[Tuple[int, int], np.ndarray]:
    """Algorithm "Belief propagation", initialisation: m = A A^H / tr(A A^H) for given
    random matrices A (one per directed edge, shape d_e x d_e)."""
    msgs = {}
    for key, a in A.items():
        p = a @ a.conj().T
        msgs[key] = p / np.trace(p)
    return msgs


_KET = "abcdefgh"
_BRA = "ABCDEFGH"


def message_update(st: VidalState, T: List[np.ndarray], msgs: Dict[Tuple[int, int], np.ndarray],
                   a: int, e: int) -> np.ndarray:
    """Eq. (local_consistency) for the message m_{a->b} along edge e = {a, b}:

    m_{a->b}[j, j'] = sum_{J, i} T_a[i, J, j] T_a^*[i, J', j'] prod_{c in da\\b} m_{c->a}[j_c, j'_c].
    """
    s = st.slot(a, e)
    k = len(st.inc[a])
    ket = "i" + _KET[:k]
    bra = "i" + _BRA[:k]
    ops = [T[a], np.conj(T[a])]
    subs = [ket, bra]
    for q, ec in enumerate(st.inc[a]):
        if q == s:
            continue
        c = st.other(ec, a)
        ops.append(msgs[directed(st, c, ec)])
        subs.append(_KET[q] + _BRA[q])
    expr = ",".join(subs) + "->" + _KET[s] + _BRA[s]
    return np.einsum(expr, *ops)


def trace_norm(A: np.ndarray) -> float:
    """||A||_1 = sum of singular values (App. C)."""
    return float(np.sum(np.linalg.svd(A, compute_uv=False)))


def bp(st: VidalState, T: List[np.ndarray], msgs: Dict[Tuple[int, int], np.ndarray],
       tol: float, max_iter: int, schedule: str = "flooding") -> Tuple[Dict, int, List[float]]:
    """Algorithm "Belief propagation" (App. B).

    Each sweep rebuilds all 2|E| messages with Eq. (local_consistency), enforces
    unit trace, and accumulates dist = sum ||m_new - m_old||_1.  The loop stops
    after the sweep in which dist/|E| < tol, or after max_iter sweeps.
    schedule="flooding" computes every new message from the previous sweep's
    messages (reading R4); "sequential" replaces messages inside the edge loop
    as the printed algorithm does.

    Returns (messages, sweeps run, [dist/|E| per sweep]).
    """
    msgs = {k: v.copy() for k, v in msgs.items()}
    hist: List[float] = []
    for it in range(1, max_iter + 1):
        dist = 0.0
        if schedule == "flooding":
            new = {}
            for e in range(st.m):
                for a in (int(st.edges[e][0]), int(st.edges[e][1])):
                    key = directed(st, a, e)
                    mm = message_update(st, T, msgs, a, e)
                    new[key] = mm / np.trace(mm)
            for key in new:
                dist += trace_norm(new[key] - msgs[key])
            msgs = new
        elif schedule == "sequential":
            for e in range(st.m):
                a, b = int(st.edges[e][0]), int(st.edges[e][1])
                mab = message_update(st, T, msgs, a, e)
                mba = message_update(st, T, msgs, b, e)
                mab = mab / np.trace(mab)
                mba = mba / np.trace(mba)
                dist += trace_norm(mab - msgs[(e, 0)])
                dist += trace_norm(mba - msgs[(e, 1)])
                msgs[(e, 0)] = mab
                msgs[(e, 1)] = mba
        else:
            raise ValueError(schedule)
        hist.append(dist / st.m if st.m else 0.0)
        if st.m == 0 or dist / st.m < tol:
            return msgs, it, hist
    return msgs, max_iter, hist


# --------------------------------------------------------------------------
# Vidal gauge from messages (App. D, Algorithm "Vidal gauge finding")
# --------------------------------------------------------------------------
def hermitian_sqrt(m: np.ndarray, eig_cutoff: float = EIG_CUTOFF) -> Tuple[np.ndarray, np.ndarray]:
    """m^{1/2} and m^{-1/2} of a Hermitian PSD message (reading R6)."""
    mh = 0.5 * (m + m.conj().T)
    w, V = np.linalg.eigh(mh)
    wmax = max(float(w.max()), 0.0)
    keep = w > eig_cutoff * wmax
    sq = np.where(keep, np.sqrt(np.where(keep, w, 0.0)), 0.0)
    isq = np.where(keep, 1.0 / np.where(keep, sq, 1.0), 0.0)
    return (V * sq) @ V.conj().T, (V * isq) @ V.conj().T


def vidal_gauge_edge(out: VidalState, e: int, msgs: Dict[Tuple[int, int], np.ndarray],
                     eig_cutoff: float = EIG_CUTOFF) -> None:
    """The loop body of Algorithm "Vidal gauge finding" for edge e = {a, b} (a = edges[e][0]):
    SVD of sum_j m^{1/2}_{a->b}[j, k] m^{1/2}_{b->a}[j, l], the two bond transforms applied
    to out.Gamma[a], out.Gamma[b] (reading R7 scaling), and lambda_ab = S / ||S||."""
    a, b = int(out.edges[e][0]), int(out.edges[e][1])
    sq_a, isq_a = hermitian_sqrt(msgs[(e, 0)], eig_cutoff)
    sq_b, isq_b = hermitian_sqrt(msgs[(e, 1)], eig_cutoff)
    M = np.einsum("jk,jl->kl", sq_a, sq_b)
    U, S, Vh = np.linalg.svd(M)
    nrm = float(np.linalg.norm(S))
    Xa = np.einsum("pq,pj->qj", isq_a, U) * np.sqrt(nrm)
    Xb = np.einsum("pq,jp->qj", isq_b, Vh) * np.sqrt(nrm)
    for x, X in ((a, Xa), (b, Xb)):
        s = out.slot(x, e)
        g = np.moveaxis(out.Gamma[x], 1 + s, -1)
        g = g @ X
        out.Gamma[x] = np.moveaxis(g, -1, 1 + s)
    out.lam[e] = S / nrm if nrm > 0 else S


def vidal_gauge(st: VidalState, T: List[np.ndarray], msgs: Dict[Tuple[int, int], np.ndarray],
                eig_cutoff: float = EIG_CUTOFF, svd_cutoff: float = SVD_CUTOFF) -> VidalState:
    """Algorithm "Vidal gauge finding" (App. D).

    Gamma_a starts as T_a.  For every edge {a, b}:
      U, lambda, V^H = SVD( sum_j m^{1/2}_{a->b}[j, k] m^{1/2}_{b->a}[j, l] ),
      Gamma_a[.., j] <- sum_{j', j''} Gamma_a[.., j''] m^{-1/2}_{a->b}[j', j''] U[j', j],
      Gamma_b[.., j] <- sum_{j', j''} Gamma_b[.., j''] m^{-1/2}_{b->a}[j', j''] V^H[j, j'].
    Reading R7 normalises lambda and scales each transform by ||S||^{1/2}; then
    zero singular values (<= svd_cutoff * s_0) are removed by Algorithm
    "Truncation".
    """
    out = VidalState(st.n, st.edges, st.inc, [t.copy() for t in T], [l.copy() for l in st.lam])
    for e in range(st.m):
        vidal_gauge_edge(out, e, msgs, eig_cutoff)
    for e in range(out.m):
        lam = out.lam[e]
        keep = int(np.sum(lam > svd_cutoff * lam[0])) if lam[0] > 0 else 1
        truncate(out, e, max(1, keep))
    return out


def local_orthogonality_residual(st: VidalState) -> float:
    """Residual R of Eq. (local_orthogonality) (App. C):

    R = 1/(2|E|) sum_a sum_{b in da} || delta - sum Gamma_a Gamma_a^* prod_{c != b} lambda_ca^2 ||_1.
    """
    if st.m == 0:
        return 0.0
    tot = 0.0
    for a in range(st.n):
        for s, e in enumerate(st.inc[a]):
            g = st.Gamma[a]
            for k, ec in enumerate(st.inc[a]):
                if k != s:
                    g = _scale_slot(g, k, st.lam[ec])
            # g carries prod_{c != b} lambda_ca once; the product with its
            # conjugate gives the lambda^2 weights of Eq. (local_orthogonality)
            g2 = np.moveaxis(g, 1 + s, -1)
            d = g2.shape[-1]
            N = g2.reshape(-1, d).T @ np.conj(g2.reshape(-1, d))
            tot += trace_norm(np.eye(d) - N)
    return tot / (2 * st.m)


# --------------------------------------------------------------------------
# marginals and read-out (Eq. partial_dens, bp_approx, rounding_rule)
# --------------------------------------------------------------------------
def reduced_density_matrices(st: VidalState, T: Optional[List[np.ndarray]] = None,
                             msgs: Optional[Dict[Tuple[int, int], np.ndarray]] = None) -> np.ndarray:
    """rho_a[i, i'] = sum T_a[i, J] T_a^*[i', J'] xi_a[J, J'] / tr, Eq. (partial_dens),
    with xi_a = prod_b m_{b->a}, Eq. (bp_approx).

    Without arguments T is the symmetric gauge of `st` and the messages are the
    warm-start messages (reading R8).  Returns an (n, 2, 2) complex array.
    """
    if T is None:
        T = symmetric_gauge(st)
    if msgs is None:
        msgs = reconstructed_messages(st)
    rho = np.zeros((st.n, 2, 2), dtype=np.complex128)
    for a in range(st.n):
        k = len(st.inc[a])
        ket = "i" + _KET[:k]
        bra = "I" + _BRA[:k]
        ops = [T[a], np.conj(T[a])]
        subs = [ket, bra]
        for q, e in enumerate(st.inc[a]):
            b = st.other(e, a)
            ops.append(msgs[directed(st, b, e)])
            subs.append(_KET[q] + _BRA[q])
        r = np.einsum(",".join(subs) + "->iI", *ops)
        rho[a] = r / np.trace(r)
    return rho


def rounding(rho: np.ndarray) -> np.ndarray:
    """Eq. (rounding_rule): x_a = +1 if rho_a[0,0] > 1/2, otherwise -1."""
    return np.where(rho[:, 0, 0].real > 0.5, 1, -1).astype(np.int8)


def objective(edges: np.ndarray, J: np.ndarray, h: np.ndarray, x: np.ndarray) -> float:
    """Eq. (objective_function): E(x) = sum J_ab x_a x_b + sum h_a x_a."""
    x = np.asarray(x, dtype=np.float64)
    return float(np.sum(J * x[edges[:, 0]] * x[edges[:, 1]]) + np.sum(h * x))


# --------------------------------------------------------------------------
# one annealing layer and a full run
# --------------------------------------------------------------------------
def gtqa_layer(st: VidalState, colour, J, h, t_Z: float, t_X: float, chi: int,
               tol: float, max_iter: int, schedule: str = "flooding",
               svd_cutoff: float = SVD_CUTOFF, eig_cutoff: float = EIG_CUTOFF,
               t_X_pre: float = 0.0) -> Tuple[VidalState, Dict]:
    """One GTQA layer: Trotter layer (gates + truncation, mixing), then regauging
    by (i) symmetric split, (ii) BP from warm-start messages, (iii) Vidal gauge
    from the messages (Sec. II C)."""
    info = trotter_layer(st, colour, J, h, t_Z, t_X, chi, svd_cutoff, t_X_pre)
    return regauge(st, tol, max_iter, schedule, svd_cutoff, eig_cutoff, info)


def regauge(st: VidalState, tol: float, max_iter: int, schedule: str = "flooding",
            svd_cutoff: float = SVD_CUTOFF, eig_cutoff: float = EIG_CUTOFF,
            info: Optional[Dict] = None) -> Tuple[VidalState, Dict]:
    """Sec. II C: symmetric split, BP from the warm-start messages, Vidal gauge from
    the converged messages."""
    info = {} if info is None else info
    T = symmetric_gauge(st)
    msgs, iters, hist = bp(st, T, reconstructed_messages(st), tol, max_iter, schedule)
    new = vidal_gauge(st, T, msgs, eig_cutoff, svd_cutoff)
    info.update({"bp_iters": iters, "bp_dist": hist[-1] if hist else 0.0, "messages": msgs, "T": T})
    return new, info


def product_formula(k: int, K: int, dt: float, order: int = 1, reverse: bool = False) -> Tuple[float, float, float]:
    """Angles (t_X_pre, t_Z, t_X_post) of layer k under reading R13 (Sec. V).

    order 1: (0, t_Z, t_X), or (t_X, t_Z, 0) when `reverse` (one draw of the randomised
    first-order formula); order 2: the symmetric formula (t_X/2, t_Z, t_X/2).
    """
    t_Z, t_X = schedule(k, K, dt)
    if order == 1:
        return (t_X, t_Z, 0.0) if reverse else (0.0, t_Z, t_X)
    if order == 2:
        if reverse:
            raise ValueError("the symmetric formula has no reversed form")
        return 0.5 * t_X, t_Z, 0.5 * t_X
    raise ValueError("order must be 1 or 2")


def apply_gates(st: VidalState, gates: Sequence[Tuple[int, np.ndarray]], chi: int,
                svd_cutoff: float = SVD_CUTOFF) -> Dict[str, float]:
    """Reading R14: arbitrary two-qubit gates (edge e, 4x4 matrix) in the order given,
    each by the simple update with truncation to chi (App. E)."""
    disc, logf = 0.0, 0.0
    for e, W in gates:
        r = simple_update(st, int(e), np.asarray(W, dtype=np.complex128).reshape(2, 2, 2, 2), chi, svd_cutoff)
        disc += r["discarded"]
        logf += np.log(r["fidelity"]) if r["fidelity"] > 0 else -np.inf
    return {"discarded": disc, "log_fidelity": logf}


def apply_single_qubit_gates(st: VidalState, gates: Sequence[Tuple[int, np.ndarray]]) -> None:
    """Sec. II D: one-qubit gates (vertex a, 2x2 matrix) in the order given."""
    for a, W in gates:
        apply_single_qubit_gate(st, int(a), np.asarray(W, dtype=np.complex128))


def run(n: int, edges, J, h, colour, K: int, dt: float, chi: int, tol: float, max_iter: int,
        layers: Optional[int] = None, record: bool = False, state: Optional[VidalState] = None,
        k0: int = 0, order: int = 1, reverse: Optional[Sequence[bool]] = None):
    """Run layers k0+1 .. k0+layers (default all K) of the anneal from |+>^N
    (or from `state`) with the product formula of reading R13 (`reverse[i]` is the
    draw of layer k0+1+i).  Returns the final state and per-layer info."""
    st = plus_state(n, np.asarray(edges)) if state is None else state
    infos = []
    last = K if layers is None else min(K, k0 + layers)
    for k in range(k0 + 1, last + 1):
        rev = bool(reverse[k - k0 - 1]) if reverse is not None else False
        t_pre, t_Z, t_X = product_formula(k, K, dt, order, rev)
        st, info = gtqa_layer(st, colour, J, h, t_Z, t_X, chi, tol, max_iter, t_X_pre=t_pre)
        if record:
            info["rho"] = reduced_density_matrices(st)
        info.pop("T", None)
        if not record:
            info.pop("messages", None)
        infos.append(info)
    return st, infos


def run_with_regauge_policy(n: int, edges, J, h, colour, K: int, dt: float, chi: int, tol: float,
                            max_iter: int, r_threshold: float, layers: Optional[int] = None,
                            state: Optional[VidalState] = None, k0: int = 0,
                            svd_cutoff: float = SVD_CUTOFF):
    """Reading R15: layers k0+1 .. k0+layers of the anneal (R1), each followed by the
    regauge of Sec. II C only when the residual R of App. C exceeds r_threshold.
    Returns the final state and per-layer {"R", "regauged"}."""
    st = plus_state(n, np.asarray(edges)) if state is None else state
    infos = []
    last = K if layers is None else min(K, k0 + layers)
    for k in range(k0 + 1, last + 1):
        t_Z, t_X = schedule(k, K, dt)
        trotter_layer(st, colour, J, h, t_Z, t_X, chi, svd_cutoff)
        R = local_orthogonality_residual(st)
        done = R > r_threshold
        if done:
            st, _ = regauge(st, tol, max_iter, svd_cutoff=svd_cutoff)
        infos.append({"R": R, "regauged": done})
    return st, infos


# --------------------------------------------------------------------------
# exact contraction of the network (tiny graphs only; used by the pins)
# --------------------------------------------------------------------------
def to_statevector(st: VidalState) -> np.ndarray:
    """Contract Eq. (vidal_gauge_tn) into the full 2^N amplitude vector (axis a = qubit a)."""
    ops: list = []
    for a in range(st.n):
        ops.append(st.Gamma[a])
        ops.append([a] + [st.n + e for e in st.inc[a]])
    for e in range(st.m):
        ops.append(st.lam[e])
        ops.append([st.n + e])
    ops.append(list(range(st.n)))
    return np.einsum(*ops, optimize="greedy")


# --------------------------------------------------------------------------
# exchange with the padded fixed-chi layout used by the CUDA library
# --------------------------------------------------------------------------
def to_padded(st: VidalState, chi: int, degree: int = 3) -> Tuple[np.ndarray, np.ndarray]:
    """Gamma as (n, 2, chi, chi, chi) and lambda as (m, chi), zero padded; vertices with
    fewer than `degree` edges get phantom slots of dimension 1 (index 0)."""
    G = np.zeros((st.n, 2) + (chi,) * degree, dtype=np.complex128)
    for a in range(st.n):
        g = st.Gamma[a]
        g = g.reshape(g.shape + (1,) * (degree - len(st.inc[a])))
        G[(a, slice(None)) + tuple(slice(0, d) for d in g.shape[1:])] = g
    L = np.zeros((st.m, chi))
    for e in range(st.m):
        L[e, :st.lam[e].size] = st.lam[e]
    return G, L


def from_padded(n: int, edges, G: np.ndarray, L: np.ndarray) -> VidalState:
    """Inverse of to_padded: bond dimensions are the number of nonzero lambda entries."""
    edges = np.asarray(edges, dtype=np.int64)
    inc = incidence(n, edges)
    lam = []
    dims = []
    for e in range(edges.shape[0]):
        d = int(np.count_nonzero(L[e]))
        d = max(d, 1)
        lam.append(np.array(L[e, :d], dtype=np.float64))
        dims.append(d)
    Gamma = []
    for a in range(n):
        k = len(inc[a])
        idx = [a, slice(None)] + [slice(0, dims[e]) for e in inc[a]] + [0] * (G.ndim - 2 - k)
        Gamma.append(np.array(G[tuple(idx)], dtype=np.complex128))
    return VidalState(n, edges, inc, Gamma, lam)


def messages_to_padded(st: VidalState, msgs: Dict[Tuple[int, int], np.ndarray], chi: int) -> np.ndarray:
    """Messages as (2m, chi, chi): row 2e is m_{u->v}, row 2e+1 is m_{v->u} for edge e = (u, v)."""
    out = np.zeros((2 * st.m, chi, chi), dtype=np.complex128)
    for (e, d), mm in msgs.items():
        out[2 * e + d, :mm.shape[0], :mm.shape[1]] = mm
    return out


def messages_from_padded(st: VidalState, P: np.ndarray) -> Dict[Tuple[int, int], np.ndarray]:
    msgs = {}
    for e in range(st.m):
        d = st.lam[e].size
        msgs[(e, 0)] = np.array(P[2 * e, :d, :d], dtype=np.complex128)
        msgs[(e, 1)] = np.array(P[2 * e + 1, :d, :d], dtype=np.complex128)
    return msgs


# --------------------------------------------------------------------------
# mean-field entanglement entropy over a bipartition (Sec. III C)
# --------------------------------------------------------------------------
def approx_entanglement_entropy(st: VidalState, cut) -> float:
    """Eq. (apprx_entropy) with the mean-field Schmidt values of Eq. (mean_field_schmidt):
    S* = - sum over the edges e of the cut of sum_j lambda_e[j]^2 log(lambda_e[j]^2).
    `cut` is a boolean (or 0/1) array over the edges; zero entries of lambda add nothing."""
    S = 0.0
    for e in range(st.m):
        if not cut[e]:
            continue
        for x in st.lam[e]:
            p = float(x) * float(x)
            if p > 0.0:
                S -= p * np.log(p)
    return S


def spectral_bipartition(n: int, edges) -> Tuple[np.ndarray, np.ndarray, float]:
    """Eq. (bipartition), A* = argmin |dA| / (|A| |Abar|), by spectral partitioning: the
    eigenvector f of the second-smallest eigenvalue of the graph Laplacian D - A (dense
    eigh), its sign fixed so that its entry of largest modulus (lowest vertex on ties) is
    positive, vertices ordered by (f, id), and the prefix of that order with the smallest
    ratio (the first one on ties).  Returns (side: True for A, cut: per edge, ratio)."""
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    L = np.zeros((n, n))
    for u, v in edges:
        L[u, v] -= 1.0
        L[v, u] -= 1.0
        L[u, u] += 1.0
        L[v, v] += 1.0
    w, V = np.linalg.eigh(L)
    f = V[:, 1].copy()
    k = int(np.argmax(np.abs(f)))
    if f[k] < 0:
        f = -f
    order = sorted(range(n), key=lambda a: (f[a], a))
    inA = np.zeros(n, dtype=bool)
    adj = [[] for _ in range(n)]
    for u, v in edges:
        adj[u].append(int(v))
        adj[v].append(int(u))
    cutsize, best, best_s = 0, np.inf, 1
    for s in range(1, n):
        u = order[s - 1]
        inside = sum(1 for x in adj[u] if inA[x])
        cutsize += len(adj[u]) - 2 * inside
        inA[u] = True
        r = cutsize / (s * (n - s))
        if r < best:
            best, best_s = r, s
    side = np.zeros(n, dtype=bool)
    side[order[:best_s]] = True
    cut = side[edges[:, 0]] != side[edges[:, 1]]
    return side, cut, float(best)


# --------------------------------------------------------------------------
# measurement sampling for degenerate problems (Sec. IV A)
# --------------------------------------------------------------------------
def sample_bitstring(st: VidalState, order, u, tol: float, max_iter: int,
                     eig_cutoff: float = EIG_CUTOFF, svd_cutoff: float = SVD_CUTOFF):
    """BP-guided sampling of a bitstring (Sec. IV A), qubit by qubit in `order`:
    (i) the outcome probabilities are the diagonal of the current reduced density matrix,
    p(x_a = +1) = rho_a[0, 0] (Eq. (partial_dens) in the Vidal gauge, reading R8); the
    outcome is +1 if u[k] < rho_a[0, 0] (u[k] uniform in [0, 1), passed in), else -1;
    (ii) Gamma_a is projected on |x_a> (Eq. (projection)); (iii) the network is regauged: BP
    from the warm start, then the Vidal gauge from the messages.
    Returns (x, p, st): x[a] in {+1, -1}, p[k] the probability of the k-th outcome given the
    previous ones, and the final state."""
    x = np.zeros(st.n, dtype=np.int8)
    p = np.zeros(len(order))
    for k, a in enumerate(order):
        rho = reduced_density_matrices(st)[a]
        p0 = float(rho[0, 0].real)
        xa = 1 if u[k] < p0 else -1
        x[a] = xa
        p[k] = p0 if xa == 1 else float(rho[1, 1].real)
        i_keep = 0 if xa == 1 else 1
        g = st.Gamma[a].copy()
        g[1 - i_keep] = 0.0
        st.Gamma[a] = g
        T = symmetric_gauge(st)
        msgs, _, _ = bp(st, T, reconstructed_messages(st), tol, max_iter)
        st = vidal_gauge(st, T, msgs, eig_cutoff, svd_cutoff)
    return x, p, st
