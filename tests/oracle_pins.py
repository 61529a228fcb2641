"""Pin checks for the CPU oracle, shared by the pin tests and the planted-mistake tests.

Every check compares the oracle with something other than itself: a matrix
exponential, the exact statevector simulation, an SVD of the exact state, a
closed-form single-qubit evolution, a symmetry, or an invariant the paper states.
Each returns the observed error (a float); the callers assert it is small.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from instances import make_instance, make_tree_instance, Instance
from oracle import gtqa_oracle as O
from oracle import statevector as SV

X = np.array([[0, 1], [1, 0]], dtype=complex)
Z = np.diag([1.0, -1.0]).astype(complex)
I2 = np.eye(2, dtype=complex)


def gate_vs_expm(seed: int = 0) -> float:
    """ising_gate / mixing_gate against scipy's expm of the defining Hamiltonians (App. F)."""
    rng = np.random.default_rng(seed)
    err = 0.0
    for _ in range(5):
        J, ha, hb, t = rng.normal(size=4)
        Da, Db = rng.integers(1, 4, size=2)
        H = J * np.kron(Z, Z) + ha / Da * np.kron(Z, I2) + hb / Db * np.kron(I2, Z)
        U = scipy.linalg.expm(-1j * t * H)
        W = O.ising_gate(J, ha, hb, int(Da), int(Db), t).reshape(4, 4)
        err = max(err, np.abs(U - W).max())
        Ux = scipy.linalg.expm(-1j * t * X)
        err = max(err, np.abs(Ux - O.mixing_gate(t)).max())
    return float(err)


def statevector_vs_dense(seed: int = 0) -> float:
    """The statevector simulator against dense expm products on K4 (n=4)."""
    rng = np.random.default_rng(seed)
    n = 4
    edges = np.array([[0, 1], [0, 2], [0, 3], [1, 2], [1, 3], [2, 3]])
    J = rng.normal(size=6)
    h = rng.normal(size=4)
    K, dt = 3, 0.4
    ops = lambda P, q: np.kron(np.kron(np.eye(2 ** q), P), np.eye(2 ** (n - q - 1)))
    H = sum(J[e] * ops(Z, a) @ ops(Z, b) for e, (a, b) in enumerate(edges)) + sum(h[a] * ops(Z, a) for a in range(n))
    HX = sum(ops(X, a) for a in range(n))
    psi = np.full(2 ** n, 2 ** (-n / 2), dtype=complex)
    for k in range(1, K + 1):
        tau = k / K
        psi = scipy.linalg.expm(-1j * dt * (1 - tau) * HX) @ (scipy.linalg.expm(-1j * dt * tau * H) @ psi)
    psi2, _ = SV.evolve(n, edges, J, h, K, dt)
    return float(np.abs(psi - psi2.reshape(-1)).max())


def _overlap_err(a: np.ndarray, b: np.ndarray) -> float:
    a = a.reshape(-1)
    b = b.reshape(-1)
    return float(abs(1 - abs(np.vdot(a, b)) / (np.linalg.norm(a) * np.linalg.norm(b))) +
                 abs(np.linalg.norm(a) - np.linalg.norm(b)))


def gates_exact_without_truncation(inst: Instance, layers: int = 2, dt: float = 0.4) -> float:
    """Trotter layers (simple update, App. E) with no truncation reproduce the
    exact state, up to a global phase (no BP, no regauge)."""
    st = O.plus_state(inst.n, inst.edges)
    K = 5
    for k in range(1, layers + 1):
        tZ, tX = O.schedule(k, K, dt)
        O.trotter_layer(st, inst.colour, inst.J, inst.h, tZ, tX, chi=1 << 12)
    psi, _ = SV.evolve(inst.n, inst.edges, inst.J, inst.h, K, dt, layers=layers, record=False)
    return _overlap_err(O.to_statevector(st), psi)


def gtqa_tree_exact(seed: int, n: int = 10, K: int = 6, dt: float = 0.3, max_degree: int = 3) -> dict:
    """On trees BP is exact (Sec. II B), so GTQA marginals without truncation equal
    the exact ones at every layer; lambda equals the edge-cut Schmidt values
    (Sec. II C); the contracted network equals the exact state.  max_degree = 4 exercises
    vertex tensors with four bonds (the 4-regular graphs of Sec. V)."""
    inst = make_tree_instance(n, seed, max_degree=max_degree)
    st = O.plus_state(inst.n, inst.edges)
    psi, rhos = SV.evolve(inst.n, inst.edges, inst.J, inst.h, K, dt)
    rho_err = 0.0
    for k in range(1, K + 1):
        tZ, tX = O.schedule(k, K, dt)
        st, info = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, 256, 1e-13, 100)
        rho_err = max(rho_err, float(np.abs(O.reduced_density_matrices(st) - rhos[k - 1]).max()))
    # Schmidt values across each edge cut
    lam_err = 0.0
    for e in range(st.m):
        a, b = inst.edges[e]
        side = _component(inst, e, int(a))
        sv = SV.schmidt_values(psi, side)
        sv = sv / np.linalg.norm(sv)
        d = st.lam[e].size
        top = sv[:d]
        lam_err = max(lam_err, float(np.abs(np.sort(st.lam[e])[::-1][:8] - top[:8]).max()))
    return {"rho": rho_err, "lam": lam_err, "state": _overlap_err(O.to_statevector(st), psi)}


def _component(inst: Instance, e_cut: int, start: int):
    adj = {a: [] for a in range(inst.n)}
    for e, (u, v) in enumerate(inst.edges.tolist()):
        if e != e_cut:
            adj[u].append(v)
            adj[v].append(u)
    seen = {start}
    stack = [start]
    while stack:
        x = stack.pop()
        for y in adj[x]:
            if y not in seen:
                seen.add(y)
                stack.append(y)
    return sorted(seen)


def gtqa_loopy_state_exact(seed: int = 0, n: int = 8, layers: int = 2, dt: float = 0.4) -> float:
    """Full GTQA layers (gates, BP, regauge) on a loopy 3-regular graph with no
    truncation: the regauge is an exact gauge transformation (App. D), so the
    contracted network still equals the exact state."""
    inst = make_instance(n, seed)
    K = 5
    st = O.plus_state(inst.n, inst.edges)
    for k in range(1, layers + 1):
        tZ, tX = O.schedule(k, K, dt)
        st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, 1 << 12, 1e-13, 200)
    psi, _ = SV.evolve(inst.n, inst.edges, inst.J, inst.h, K, dt, layers=layers, record=False)
    return _overlap_err(O.to_statevector(st), psi)


def product_state_closed_form(seed: int = 0, n: int = 16, K: int = 12, dt: float = 0.3) -> float:
    """J = 0: the state stays a product state; each qubit follows the 2x2 evolution
    prod_k exp(-i t_X X) exp(-i t_Z h_a Z) applied to |+> (closed form)."""
    inst = make_instance(n, seed)
    inst.J[:] = 0.0
    st = O.plus_state(inst.n, inst.edges)
    err = 0.0
    for k in range(1, K + 1):
        tZ, tX = O.schedule(k, K, dt)
        st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, 4, 1e-13, 100)
        rho = O.reduced_density_matrices(st)
        for a in range(n):
            v = np.array([1, 1], dtype=complex) / np.sqrt(2)
            for q in range(1, k + 1):
                tz, tx = O.schedule(q, K, dt)
                v = np.diag(np.exp(-1j * tz * inst.h[a] * np.array([1, -1]))) @ v
                v = np.array([[np.cos(tx), -1j * np.sin(tx)], [-1j * np.sin(tx), np.cos(tx)]]) @ v
            err = max(err, float(np.abs(rho[a] - np.outer(v, v.conj())).max()))
        err = max(err, float(max(l.size for l in st.lam) - 1))
    return err


def z2_symmetry(seed: int = 0, n: int = 16, K: int = 20, dt: float = 0.1, chi: int = 4) -> float:
    """h = 0: prod_a X_a commutes with H(t) and |+>^N is symmetric, so <Z_a> = 0 exactly."""
    inst = make_instance(n, seed, h_std=0.0)
    st = O.plus_state(inst.n, inst.edges)
    err = 0.0
    for k in range(1, K + 1):
        tZ, tX = O.schedule(k, K, dt)
        st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, chi, 1e-12, 100)
        rho = O.reduced_density_matrices(st)
        err = max(err, float(np.abs(rho[:, 0, 0].real - 0.5).max()))
    return err


def loopy_state(seed: int = 0, n: int = 16, layers: int = 5, K: int = 20, dt: float = 0.1, chi: int = 4):
    inst = make_instance(n, seed)
    st = O.plus_state(inst.n, inst.edges)
    for k in range(1, layers + 1):
        tZ, tX = O.schedule(k, K, dt)
        st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, chi, 1e-13, 100)
    return inst, st


def after_gates(seed: int = 0, n: int = 16, layers: int = 5, K: int = 20, dt: float = 0.1, chi: int = 4):
    """A loopy state right after a Trotter layer (Vidal gauge broken by truncation)."""
    inst, st = loopy_state(seed, n, layers, K, dt, chi)
    tZ, tX = O.schedule(layers + 1, K, dt)
    O.trotter_layer(st, inst.colour, inst.J, inst.h, tZ, tX, chi)
    return inst, st


def bp_gauge_covariance(seed: int = 0) -> float:
    """Inserting an invertible G and G^{-T} on every bond of T leaves the network (and
    so the BP fixed point's marginals) unchanged: checks the index placement of
    Eq. (local_consistency) and Eq. (partial_dens)."""
    inst, st = after_gates(seed)
    rng = np.random.default_rng(seed)
    T = O.symmetric_gauge(st)
    T2 = [t.copy() for t in T]
    for e in range(st.m):
        d = st.lam[e].size
        G = np.eye(d) + 0.3 * (rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d)))
        Gi = np.linalg.inv(G).T
        for x, M in ((int(inst.edges[e][0]), G), (int(inst.edges[e][1]), Gi)):
            s = st.slot(x, e)
            g = np.moveaxis(T2[x], 1 + s, -1) @ M
            T2[x] = np.moveaxis(g, -1, 1 + s)
    A = {}
    for e in range(st.m):
        d = st.lam[e].size
        for dd in (0, 1):
            A[(e, dd)] = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    m1, _, _ = O.bp(st, T, O.random_messages(st, A), 1e-14, 400)
    m2, _, _ = O.bp(st, T2, O.random_messages(st, A), 1e-14, 400)
    r1 = O.reduced_density_matrices(st, T, m1)
    r2 = O.reduced_density_matrices(st, T2, m2)
    return float(np.abs(r1 - r2).max())


def bp_invariants(seed: int = 0) -> float:
    """Messages are Hermitian, positive semi-definite and of unit trace (Sec. II B, App. B)."""
    inst, st = after_gates(seed)
    T = O.symmetric_gauge(st)
    msgs, _, _ = O.bp(st, T, O.reconstructed_messages(st), 1e-12, 100)
    err = 0.0
    for mm in msgs.values():
        err = max(err, float(np.abs(mm - mm.conj().T).max()))
        err = max(err, float(abs(np.trace(mm) - 1)))
        err = max(err, float(max(0.0, -np.linalg.eigvalsh(0.5 * (mm + mm.conj().T)).min())))
    return err


def flooding_vs_sequential(seed: int = 0) -> float:
    """Both schedules solve the same fixed-point equation, Eq. (local_consistency)."""
    inst, st = after_gates(seed)
    T = O.symmetric_gauge(st)
    m1, _, _ = O.bp(st, T, O.reconstructed_messages(st), 1e-14, 300, "flooding")
    m2, _, _ = O.bp(st, T, O.reconstructed_messages(st), 1e-14, 300, "sequential")
    return float(np.abs(O.reduced_density_matrices(st, T, m1) - O.reduced_density_matrices(st, T, m2)).max())


def warm_start_fixed_point(seed: int = 0) -> float:
    """After regauging (R = 0) the warm-start messages solve Eq. (local_consistency):
    one BP sweep changes them by nothing (Sec. II C)."""
    inst, st = loopy_state(seed)
    T = O.symmetric_gauge(st)
    _, it, hist = O.bp(st, T, O.reconstructed_messages(st), 0.0, 1)
    return float(hist[0])


def residual_after_regauge(seed: int = 0) -> float:
    """The Vidal gauge found from converged messages has R = 0 (App. C-D)."""
    inst, st = loopy_state(seed)
    return O.local_orthogonality_residual(st)


def regauge_is_exact_gauge_transform(seed: int = 0) -> float:
    """Algorithm "Vidal gauge finding" changes only the gauge: the contracted state
    is unchanged (loopy 3-regular graph, n = 8, truncated state)."""
    inst = make_instance(8, seed)
    st = O.plus_state(inst.n, inst.edges)
    K, dt = 10, 0.3
    for k in range(1, 4):
        tZ, tX = O.schedule(k, K, dt)
        st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, 2, 1e-13, 200)
    tZ, tX = O.schedule(4, K, dt)
    O.trotter_layer(st, inst.colour, inst.J, inst.h, tZ, tX, 2)
    before = O.to_statevector(st)
    T = O.symmetric_gauge(st)
    msgs, _, _ = O.bp(st, T, O.reconstructed_messages(st), 1e-14, 300)
    new = O.vidal_gauge(st, T, msgs)
    after = O.to_statevector(new)
    return float(np.abs(before - after).max() / np.abs(before).max())


def truncation_frobenius(seed: int = 0) -> float:
    """Truncating the smallest Schmidt values of one edge of a tree in the Vidal
    gauge moves the state by exactly sqrt(sum of dropped lambda^2) (Sec. II C)."""
    inst = make_tree_instance(10, seed)
    st = O.plus_state(inst.n, inst.edges)
    K, dt = 6, 0.3
    for k in range(1, 5):
        tZ, tX = O.schedule(k, K, dt)
        st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, 256, 1e-13, 100)
    psi = O.to_statevector(st)
    err = 0.0
    for e in range(st.m):
        d = st.lam[e].size
        if d < 3:
            continue
        cut = O.VidalState(st.n, st.edges, st.inc, [g.copy() for g in st.Gamma], [l.copy() for l in st.lam])
        dropped = st.lam[e][d - 1:]
        O.truncate(cut, e, d - 1)
        dpsi = np.linalg.norm(psi - O.to_statevector(cut))
        err = max(err, abs(dpsi - np.sqrt(np.sum(dropped ** 2))))
    return float(err)


def single_edge_exact(seed: int = 0) -> float:
    """n = 2, one edge: the Schmidt rank is at most 2, so GTQA is exact at chi = 2."""
    rng = np.random.default_rng(seed)
    edges = np.array([[0, 1]])
    J = rng.normal(size=1)
    h = rng.normal(size=2)
    colour = np.zeros(1, dtype=np.int32)
    K, dt = 10, 0.5
    st = O.plus_state(2, edges)
    psi, rhos = SV.evolve(2, edges, J, h, K, dt)
    err = 0.0
    for k in range(1, K + 1):
        tZ, tX = O.schedule(k, K, dt)
        st, _ = O.gtqa_layer(st, colour, J, h, tZ, tX, 2, 1e-13, 100)
        err = max(err, float(np.abs(O.reduced_density_matrices(st) - rhos[k - 1]).max()))
    return err


def trace_distance_band(seeds=(0, 1, 2), n: int = 14, T: float = 20.0, dt: float = 0.2, chi: int = 4) -> float:
    """Eq. (error): qubit- and time-averaged trace distance between BP and exact
    marginals.  The paper reports 1e-3 .. a few 1e-2 at N = 14..26, T = 20, chi = 4."""
    K = int(round(T / dt))
    errs = []
    for s in seeds:
        inst = make_instance(n, s)
        st = O.plus_state(inst.n, inst.edges)
        _, rhos = SV.evolve(inst.n, inst.edges, inst.J, inst.h, K, dt)
        tot = 0.0
        for k in range(1, K + 1):
            tZ, tX = O.schedule(k, K, dt)
            st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, chi, 1e-10, 100)
            rho = O.reduced_density_matrices(st)
            for a in range(n):
                tot += O.trace_norm(rho[a] - rhos[k - 1][a])
        errs.append(dt / (2 * T * n) * tot)
    return float(np.mean(errs))


def tree_entropy_exact(seed: int, n: int = 10, K: int = 5, dt: float = 0.3) -> float:
    """On a tree without truncation, lambda across an edge are the Schmidt values of that
    edge's cut (Sec. II C), so the mean-field entropy of Eq. (apprx_entropy) for a one-edge
    cut equals the von Neumann entropy of the exact state for that bipartition."""
    inst = make_tree_instance(n, seed)
    st = O.plus_state(inst.n, inst.edges)
    psi, _ = SV.evolve(inst.n, inst.edges, inst.J, inst.h, K, dt)
    for k in range(1, K + 1):
        tZ, tX = O.schedule(k, K, dt)
        st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, 256, 1e-13, 100)
    err = 0.0
    for e in range(st.m):
        side = _component(inst, e, int(inst.edges[e][0]))
        sv = SV.schmidt_values(psi, side)
        p = (sv / np.linalg.norm(sv)) ** 2
        p = p[p > 1e-300]
        s_exact = float(-(p * np.log(p)).sum())
        cut = np.zeros(st.m, dtype=bool)
        cut[e] = True
        err = max(err, abs(O.approx_entanglement_entropy(st, cut) - s_exact))
    return err


def bipartition_closed_forms() -> float:
    """Eq. (bipartition) on graphs whose best ratio cut is known: two 4-cliques joined by
    one edge (the cliques, ratio 1/16) and the 12-cycle (two arcs of 6, ratio 2/36); the
    spectral split must find them.  Returns the largest deviation of the ratio."""
    err = 0.0
    k4 = [(a, b) for a in range(4) for b in range(a + 1, 4)]
    edges = np.array(k4 + [(a + 4, b + 4) for a, b in k4] + [(3, 4)])
    side, cut, r = O.spectral_bipartition(8, edges)
    err = max(err, abs(r - 1 / 16), float(abs(int(cut.sum()) - 1)))
    err = max(err, float(len({bool(side[a]) for a in range(4)}) - 1))
    ring = np.array([(a, (a + 1) % 12) for a in range(12)])
    side, cut, r = O.spectral_bipartition(12, ring)
    err = max(err, abs(r - 2 / 36), float(abs(int(cut.sum()) - 2)))
    return float(err)


def bipartition_against_brute_force(seed: int = 0, n: int = 12) -> float:
    """The spectral split is a heuristic for Eq. (bipartition): on small random 3-regular
    graphs its ratio is never below the exhaustive minimum over all 2^(n-1) - 1 splits, and
    the reported cut and ratio are consistent with the returned sides."""
    inst = make_instance(n, seed)
    side, cut, r = O.spectral_bipartition(n, inst.edges)
    e = inst.edges
    best = np.inf
    for mask in range(1, 2 ** (n - 1)):
        s = np.array([(mask >> a) & 1 for a in range(n)], dtype=bool)
        c = int((s[e[:, 0]] != s[e[:, 1]]).sum())
        best = min(best, c / (s.sum() * (n - s.sum())))
    consistent = abs(r - int(cut.sum()) / (side.sum() * (n - side.sum())))
    below = max(0.0, best - r)
    return float(max(consistent, below))


def tree_sampling_chain_rule(seed: int, n: int = 8, K: int = 4, dt: float = 0.4) -> float:
    """Measurement sampling (Sec. IV A) on a tree without truncation: BP marginals are exact
    (Sec. II B), so the product of the conditional probabilities of a sampled bitstring is
    its exact Born probability |<x|psi>|^2 from the statevector.  Returns the relative error."""
    inst = make_tree_instance(n, seed)
    st = O.plus_state(inst.n, inst.edges)
    psi, _ = SV.evolve(inst.n, inst.edges, inst.J, inst.h, K, dt)
    for k in range(1, K + 1):
        tZ, tX = O.schedule(k, K, dt)
        st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, 256, 1e-13, 100)
    rng = np.random.default_rng(100 + seed)
    order = rng.permutation(n).tolist()
    u = rng.random(n)
    x, p, _ = O.sample_bitstring(st, order, u, 1e-13, 100)
    idx = tuple(0 if xa == 1 else 1 for xa in x)
    born = abs(psi[idx]) ** 2 / np.sum(np.abs(psi) ** 2)
    return float(abs(np.prod(p) - born) / born)


# --------------------------------------------------------------------------
# product formulas and arbitrary gates (Sec. V; Sec. II D, App. E)
# --------------------------------------------------------------------------
def _one_layer_error(n, edges, J, h, tau, dt, order, mode):
    """Distance after one layer from |+>^n between the product formula and
    expm(-i dt (tau H_Z + (1 - tau) H_X)).  mode "fwd"/"rev" compares states, mode "avg"
    compares the density matrix averaged over the two orderings (randomised formula)."""
    E = SV.interaction_phase(n, edges, J, h).reshape(-1)
    ops = lambda P, q: np.kron(np.kron(np.eye(2 ** q), P), np.eye(2 ** (n - q - 1)))
    HX = sum(ops(X, a) for a in range(n))
    U = scipy.linalg.expm(-1j * dt * (tau * np.diag(E) + (1 - tau) * HX))
    psi0 = np.full(2 ** n, 2 ** (-n / 2), dtype=complex)
    exact = U @ psi0
    K = 10
    k = int(round(tau * K))
    dt_l = dt

    def layer(rev):
        ang = O.product_formula(k, K, dt_l, order, rev)
        psi, _ = SV.evolve_split(n, edges, J, h, [ang], record=False)
        return psi.reshape(-1)

    if mode == "avg":
        pf, pr = layer(False), layer(True)
        rho = 0.5 * (np.outer(pf, pf.conj()) + np.outer(pr, pr.conj()))
        return float(np.linalg.norm(rho - np.outer(exact, exact.conj())))
    psi = layer(mode == "rev")
    return float(np.linalg.norm(psi - exact))


def product_formula_orders(seed: int = 0) -> dict:
    """Local error of one layer against the matrix exponential of the layer's
    Hamiltonian (reading R13): the first-order formula (either ordering) errs by O(dt^2),
    the symmetric formula and the average over the two first-order orderings (the
    randomised formula, as a channel) by O(dt^3).  Returns e(dt)/e(dt/2) per formula
    (about 4 and 8)."""
    inst = make_instance(6, seed)
    out = {}
    for name, order, mode in (("first", 1, "fwd"), ("first_rev", 1, "rev"), ("second", 2, "fwd"),
                              ("randomised", 1, "avg")):
        e1 = _one_layer_error(inst.n, inst.edges, inst.J, inst.h, 0.4, 0.08, order, mode)
        e2 = _one_layer_error(inst.n, inst.edges, inst.J, inst.h, 0.4, 0.04, order, mode)
        out[name] = e1 / e2
    return out


def tree_product_formula_exact(seed: int, order: int, n: int = 10, K: int = 6, dt: float = 0.3) -> float:
    """On a tree without truncation the GTQA marginals under the second-order or the
    randomised first-order formula equal the exact ones layer by layer (Sec. II B, R13)."""
    inst = make_tree_instance(n, seed)
    rng = np.random.default_rng(seed + 99)
    rev = [bool(x) for x in rng.integers(0, 2, size=K)] if order == 1 else [False] * K
    angles = [O.product_formula(k, K, dt, order, rev[k - 1]) for k in range(1, K + 1)]
    _, rhos = SV.evolve_split(inst.n, inst.edges, inst.J, inst.h, angles)
    st = O.plus_state(inst.n, inst.edges)
    err = 0.0
    for k in range(1, K + 1):
        t_pre, tZ, tX = angles[k - 1]
        st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, 256, 1e-13, 100, t_X_pre=t_pre)
        err = max(err, float(np.abs(O.reduced_density_matrices(st) - rhos[k - 1]).max()))
    return err


def random_unitary(rng: np.random.Generator, d: int) -> np.ndarray:
    """Haar-distributed d x d unitary (QR of a complex Gaussian matrix with the phases of
    R's diagonal divided out)."""
    A = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    Q, R = np.linalg.qr(A)
    return Q * (np.diag(R) / np.abs(np.diag(R)))[None, :]


def random_gate_list(rng: np.random.Generator, m: int, k: int):
    """k gates on uniformly drawn edges (repeats allowed), Haar 4x4 unitaries."""
    return [(int(rng.integers(m)), random_unitary(rng, 4)) for _ in range(k)]


def general_gates_exact(seed: int = 0, n: int = 8, k: int = 14) -> dict:
    """Arbitrary two- and one-qubit gates on a tree without truncation reproduce the
    exact state (reading R14); after the regauge (exact BP on a tree) the marginals are
    the exact ones."""
    inst = make_tree_instance(n, seed)
    rng = np.random.default_rng(seed + 7)
    st = O.plus_state(inst.n, inst.edges)
    psi = SV.plus_state(inst.n)
    for rnd in range(2):
        gates = random_gate_list(rng, inst.m, k)
        singles = [(int(rng.integers(inst.n)), random_unitary(rng, 2)) for _ in range(n)]
        O.apply_gates(st, gates, 256)
        O.apply_single_qubit_gates(st, singles)
        for e, W in gates:
            a, b = (int(x) for x in inst.edges[e])
            psi = SV.apply_two(psi, a, b, W)
        for a, W in singles:
            psi = SV.apply_one(psi, a, W)
    state_err = _overlap_err(O.to_statevector(st), psi)
    new, _ = O.regauge(st, 1e-13, 200)
    rho_err = float(np.abs(O.reduced_density_matrices(new) - SV.all_rdm1(psi)).max())
    return {"state": state_err, "rho": rho_err}


def general_gate_truncation_fidelity(seed: int = 0, n: int = 10) -> float:
    """On a tree in the Vidal gauge, one arbitrary gate followed by truncation to chi keeps
    the optimal rank-chi Schmidt approximation: w, the discarded weight, is the weight of
    the smallest exact Schmidt values across the edge, and |<psi|psi_trunc>|^2 = 1 - w
    (Sec. II C, App. E, Eq. (gate_fidelity))."""
    inst = make_tree_instance(n, seed)
    rng = np.random.default_rng(seed + 3)
    st = O.plus_state(inst.n, inst.edges)
    O.apply_gates(st, random_gate_list(rng, inst.m, 3 * inst.m), 256)
    st, _ = O.regauge(st, 1e-14, 300)
    err = 0.0
    for e in range(inst.m):
        d = st.lam[e].size
        if d < 2:
            continue
        W = random_unitary(rng, 4)
        ref = O.VidalState(st.n, st.edges, st.inc, [g.copy() for g in st.Gamma], [l.copy() for l in st.lam])
        O.apply_gates(ref, [(e, W)], 256)
        cut = O.VidalState(st.n, st.edges, st.inc, [g.copy() for g in st.Gamma], [l.copy() for l in st.lam])
        r = O.apply_gates(cut, [(e, W)], max(1, ref.lam[e].size - 1))
        psi = O.to_statevector(ref)
        a = psi.reshape(-1)
        b = O.to_statevector(cut).reshape(-1)
        ov = abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)
        # the discarded weight is that of the smallest exact Schmidt values across e
        sv = SV.schmidt_values(psi / np.linalg.norm(a), _component(inst, e, int(inst.edges[e][0])))
        w_opt = float(np.sum(sv[ref.lam[e].size - 1:] ** 2))
        err = max(err, abs(ov - (1.0 - r["discarded"])), abs(r["discarded"] - w_opt))
    return float(err)


def regauge_policy_on_trees(seed: int = 0, n: int = 10, K: int = 6, dt: float = 0.3) -> dict:
    """Reading R15 on a tree without truncation: the simple update is exact there (Sec. II B-C),
    so a policy that never regauges (infinite threshold) still gives the exact marginals at
    every layer, and so does one that always regauges."""
    inst = make_tree_instance(n, seed)
    _, rhos = SV.evolve(inst.n, inst.edges, inst.J, inst.h, K, dt)
    out = {}
    for name, thr in (("never", np.inf), ("always", -1.0)):
        st = None
        err = 0.0
        regauged = 0
        for k in range(1, K + 1):
            st, infos = O.run_with_regauge_policy(inst.n, inst.edges, inst.J, inst.h, inst.colour, K, dt, 256, 1e-13,
                                                  100, thr, layers=1, state=st, k0=k - 1)
            regauged += sum(i["regauged"] for i in infos)
            err = max(err, float(np.abs(O.reduced_density_matrices(st) - rhos[k - 1]).max()))
        out[name] = {"regauged": regauged, "rho": err}
    return out


def regauge_policy_on_loopy_graphs(seed: int = 0, n: int = 16, K: int = 20, dt: float = 0.1, chi: int = 4) -> dict:
    """On a loopy graph with truncation: a negative threshold regauges every layer and is the
    every-layer run (reading R1); an infinite one never regauges; at an intermediate threshold
    exactly the layers whose R exceeds it are regauged."""
    inst = make_instance(n, seed)
    layers = 6
    args = (inst.n, inst.edges, inst.J, inst.h, inst.colour, K, dt, chi, 1e-12, 100)
    st_a, infos_a = O.run_with_regauge_policy(*args, -1.0, layers=layers)
    st_b, _ = O.run(*args, layers=layers)
    _, infos_c = O.run_with_regauge_policy(*args, np.inf, layers=layers)
    Rs = sorted(i["R"] for i in infos_a)
    thr = 0.5 * (Rs[len(Rs) // 2 - 1] + Rs[len(Rs) // 2])
    _, infos_d = O.run_with_regauge_policy(*args, thr, layers=layers)
    return {"all_regauged": all(i["regauged"] for i in infos_a),
            "rho": float(np.abs(O.reduced_density_matrices(st_a) - O.reduced_density_matrices(st_b)).max()),
            "none_regauged": not any(i["regauged"] for i in infos_c),
            "threshold_rule": all(i["regauged"] == (i["R"] > thr) for i in infos_d),
            "some_skipped": 0 < sum(i["regauged"] for i in infos_d) < layers}


def residual_closed_form() -> float:
    """R of App. C on a hand-built 3-vertex path 0 - 1 - 2 (edges e0 = (0, 1), e1 = (1, 2)) whose
    value follows by hand.  lambda_e0 = (cos 0.3, sin 0.3), lambda_e1 = (cos 0.7, sin 0.7);
    Gamma_0[i, j0] = diag(sqrt(1 + 0.05), sqrt(1 - 0.02)); Gamma_2 = identity; Gamma_1[i, j0, j1]
    = delta(i, j0) c[j1].  Per directed bond the matrix sum_rest Gamma Gamma^* prod_{other} lambda^2
    is: at vertex 0, diag(1.05, 0.98) (trace norm of I minus it: 0.07); at vertex 2, I (0); at
    vertex 1 on e0, s I with s = |c0|^2 cos^2 0.7 + |c1|^2 sin^2 0.7 (2 |1 - s|); at vertex 1 on
    e1, c c^H, since sum_i lambda_e0[i]^2 = 1 (eigenvalues |c|^2 and 0, so |1 - |c|^2| + 1).
    R divides the sum by 2|E| = 4.  Returns |oracle R - closed form|."""
    a, b = 0.3, 0.7
    c = np.array([0.8 + 0.1j, 0.3 - 0.4j])
    edges = np.array([[0, 1], [1, 2]], dtype=np.int64)
    inc = O.incidence(3, edges)
    G0 = np.diag([np.sqrt(1.05), np.sqrt(0.98)]).astype(np.complex128)
    G2 = np.eye(2, dtype=np.complex128)
    G1 = np.zeros((2, 2, 2), dtype=np.complex128)
    for i in range(2):
        G1[i, i, :] = c
    lam = [np.array([np.cos(a), np.sin(a)]), np.array([np.cos(b), np.sin(b)])]
    st = O.VidalState(3, edges, inc, [G0, G1, G2], lam)
    s = abs(c[0]) ** 2 * np.cos(b) ** 2 + abs(c[1]) ** 2 * np.sin(b) ** 2
    c2 = float(np.sum(np.abs(c) ** 2))
    closed = (0.07 + 0.0 + 2 * abs(1 - s) + abs(1 - c2) + 1.0) / 4.0
    return abs(O.local_orthogonality_residual(st) - closed)
