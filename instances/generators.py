"""Seeded instance generators: random d-regular graphs, random trees, Gaussian
Ising couplings and fields, and a proper edge colouring (disjoint matchings).

Workload shape follows the paper's QUBO benchmark (Sec. III B): random
3-regular graphs with couplings J_ab and fields h_a drawn from normal
distributions.  The paper samples graphs with the Steger-Wormald algorithm;
here the configuration (pairing) model with rejection is used, which samples
simple d-regular graphs uniformly.  All randomness comes from numpy's PCG64
seeded explicitly, so every instance is reproducible from its seed.

The edge colouring is a schedule input, not part of the paper's method: the
paper applies the two-qubit gates of the interaction layer "sequentially"
without fixing an order (Sec. III A, App. F).  Gates of one colour act on
disjoint vertex pairs, so they commute and may run in one launch.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Tuple

import numpy as np

BASE_SEED = 2409122400


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def random_regular_graph(n: int, d: int, seed: int, max_tries: int = 10000) -> np.ndarray:
    """Uniform simple d-regular graph on n vertices (pairing model + rejection).

    Returns an (m, 2) int32 array of edges (u < v), sorted lexicographically,
    m = n d / 2.
    """
    if (n * d) % 2 != 0 or d >= n:
        raise ValueError("n*d must be even and d < n")
    rng = _rng(seed)
    points = np.repeat(np.arange(n, dtype=np.int64), d)
    for _ in range(max_tries):
        perm = rng.permutation(points)
        u = perm[0::2]
        v = perm[1::2]
        if np.any(u == v):
            continue
        a = np.minimum(u, v)
        b = np.maximum(u, v)
        key = a * n + b
        if np.unique(key).size != key.size:
            continue
        order = np.argsort(key)
        return np.stack([a[order], b[order]], axis=1).astype(np.int32)
    raise RuntimeError("pairing model failed to produce a simple graph")


def random_tree(n: int, seed: int, max_degree: int = 3) -> np.ndarray:
    """Random tree on n vertices with maximum degree max_degree.

    Vertex k (k >= 1) attaches to a uniformly chosen earlier vertex that still
    has spare degree.  Returns sorted (m, 2) int32 edges with m = n - 1.
    """
    rng = _rng(seed)
    deg = np.zeros(n, dtype=np.int64)
    edges = []
    for k in range(1, n):
        cand = np.nonzero(deg[:k] < max_degree)[0]
        p = int(cand[rng.integers(cand.size)])
        edges.append((p, k))
        deg[p] += 1
        deg[k] += 1
    e = np.array(sorted(edges), dtype=np.int32).reshape(-1, 2)
    return e


def heavy_hex_graph(rows: int, cols: int) -> Tuple[int, np.ndarray]:
    """Heavy-hexagon lattice (the degree-2/3 qubit layout of Sec. V's loop study):
    `rows` chains of `cols` vertices each, and between chains r and r+1 a bridge vertex
    joined to both chains at every column c with c = 2 (r mod 2) (mod 4).  Bridges
    above and below a chain sit at columns 2 apart, so every vertex has degree <= 3,
    every cycle is even, and the shortest cycles (one hexagon: 4 + 4 chain edges, 2 + 2
    bridge edges) have length 12.  Returns (n, sorted (m, 2) int32 edges)."""
    if rows < 1 or cols < 1:
        raise ValueError("rows and cols must be positive")
    vid = lambda r, c: r * cols + c
    n = rows * cols
    edges = []
    for r in range(rows):
        for c in range(cols - 1):
            edges.append((vid(r, c), vid(r, c + 1)))
    for r in range(rows - 1):
        for c in range(2 * (r % 2), cols, 4):
            b = n
            n += 1
            edges.append((vid(r, c), b))
            edges.append((vid(r + 1, c), b))
    e = np.array(sorted((min(u, v), max(u, v)) for u, v in edges), dtype=np.int32).reshape(-1, 2)
    return n, e


def edge_colouring(n: int, edges: np.ndarray, seed: int = 0) -> np.ndarray:
    """Proper edge colouring, each colour class a matching: Delta colours when the Kempe-chain
    search below finds them (almost all random cubic graphs, trees and heavy-hexagon lattices
    are Delta-edge-colourable), else Misra-Gries with at most Delta + 1.  Fewer colours means
    fewer sequential gate phases per layer.  Returns an int32 array colour[e]."""
    col = delta_edge_colouring(n, edges, seed)
    return col if col is not None else misra_gries_colouring(n, edges)


def delta_edge_colouring(n: int, edges: np.ndarray, seed: int = 0,
                         max_steps: Optional[int] = None) -> Optional[np.ndarray]:
    """Try to colour the edges with Delta = max degree colours; None if the search gives up.

    Edges are coloured in a seeded random order.  An edge {u, v} takes a colour free at both
    ends if there is one.  Otherwise, with a free at u and b free at v, the a/b Kempe chain that
    starts at v is swapped, which frees a at v, unless the chain ends at u (it would close an
    odd cycle with {u, v}).  In that case a random Kempe component through u or v is swapped,
    which keeps the colouring proper, and the edge is tried again.  The search gives up after
    max_steps attempts (default 200 m + 1000)."""
    edges = np.asarray(edges, dtype=np.int64)
    m = int(edges.shape[0])
    if m == 0:
        return np.zeros(0, dtype=np.int32)
    D = int(np.bincount(edges.ravel(), minlength=n).max())
    if D == 1:
        return np.zeros(m, dtype=np.int32)
    rng = _rng(BASE_SEED + 9_000_000 + int(seed))
    E = edges.tolist()
    at = np.full((n, D), -1, dtype=np.int64)     # edge of colour c at vertex v
    col = np.full(m, -1, dtype=np.int64)

    def other(f, x):
        return E[f][0] if E[f][1] == x else E[f][1]

    def recolour(fs, a, b):
        for f in fs:
            p, q = E[f]
            at[p, col[f]] = -1
            at[q, col[f]] = -1
        for f in fs:
            col[f] = b if col[f] == a else a
            p, q = E[f]
            at[p, col[f]] = f
            at[q, col[f]] = f

    def component(x, a, b):
        comp, seen, stack, visited = [], set(), [x], {x}
        while stack:
            y = stack.pop()
            for c in (a, b):
                f = int(at[y, c])
                if f >= 0 and f not in seen:
                    seen.add(f)
                    comp.append(f)
                    z = other(f, y)
                    if z not in visited:
                        visited.add(z)
                        stack.append(z)
        return comp

    steps, limit = 0, (max_steps if max_steps is not None else 200 * m + 1000)
    for e in rng.permutation(m).tolist():
        u, v = E[e]
        while True:
            steps += 1
            if steps > limit:
                return None
            fu = [c for c in range(D) if at[u, c] < 0]
            fv = [c for c in range(D) if at[v, c] < 0]
            common = [c for c in fu if c in fv]
            if common:
                c = common[int(rng.integers(len(common)))]
                break
            a = fu[int(rng.integers(len(fu)))]
            b = fv[int(rng.integers(len(fv)))]
            path, x, cc = [], v, a
            while at[x, cc] >= 0:
                f = int(at[x, cc])
                path.append(f)
                x = other(f, x)
                cc = b if cc == a else a
            if x != u:
                recolour(path, a, b)
                c = a
                break
            p, q = (int(t) for t in rng.choice(D, size=2, replace=False))
            recolour(component((u, v)[int(rng.integers(2))], p, q), p, q)
        col[e] = c
        at[u, c] = e
        at[v, c] = e
    return col.astype(np.int32)


def misra_gries_colouring(n: int, edges: np.ndarray) -> np.ndarray:
    """Proper edge colouring with at most Delta+1 colours (Misra-Gries).

    Returns an int32 array colour[e]; edges sharing a vertex get different
    colours, so each colour class is a matching.
    """
    edges = np.asarray(edges, dtype=np.int64)
    m = edges.shape[0]
    deg = np.bincount(edges.ravel(), minlength=n) if m else np.zeros(n, dtype=np.int64)
    ncol = int(deg.max()) + 1 if m else 1
    # at[v][c] = neighbour reached from v by the edge of colour c (or -1)
    at = np.full((n, ncol), -1, dtype=np.int64)
    eid = {}
    for k, (u, v) in enumerate(edges):
        eid[(int(u), int(v))] = k
        eid[(int(v), int(u))] = k
    colour = np.full(m, -1, dtype=np.int64)

    def free(v):
        for c in range(ncol):
            if at[v, c] < 0:
                return c
        raise RuntimeError("no free colour")

    def is_free(v, c):
        return at[v, c] < 0

    def set_col(u, v, c):
        k = eid[(u, v)]
        old = colour[k]
        if old >= 0:
            at[u, old] = -1
            at[v, old] = -1
        colour[k] = c
        if c >= 0:
            at[u, c] = v
            at[v, c] = u

    for k, (u0, v0) in enumerate(edges):
        u, v = int(u0), int(v0)
        # maximal fan of u starting at v
        fan = [v]
        used = {v}
        while True:
            last = fan[-1]
            nxt = None
            for c in range(ncol):
                if is_free(last, c):
                    w = at[u, c]
                    if w >= 0 and w not in used:
                        nxt = int(w)
                        break
            if nxt is None:
                break
            fan.append(nxt)
            used.add(nxt)
        c = free(u)
        dcol = free(fan[-1])
        # invert the cd-path starting at u
        if not is_free(u, dcol):
            path = [u]
            cur, col = u, dcol
            while at[cur, col] >= 0:
                nxt = int(at[cur, col])
                path.append(nxt)
                cur = nxt
                col = c if col == dcol else dcol
            pedges = [(path[i], path[i + 1]) for i in range(len(path) - 1)]
            pcols = [colour[eid[e]] for e in pedges]
            for e in pedges:
                set_col(e[0], e[1], -1)
            for e, pc in zip(pedges, pcols):
                set_col(e[0], e[1], dcol if pc == c else c)
        # find w in the fan with d free; rotate the fan up to w
        widx = None
        for i, w in enumerate(fan):
            if is_free(w, dcol):
                ok = True
                # the prefix fan[0..i] must still be a fan after the inversion
                for j in range(1, i + 1):
                    cj = colour[eid[(u, fan[j])]]
                    if cj < 0 or not is_free(fan[j - 1], cj):
                        ok = False
                        break
                if ok:
                    widx = i
                    break
        if widx is None:
            raise RuntimeError("Misra-Gries: no valid fan prefix")
        for j in range(widx):
            cj = colour[eid[(u, fan[j + 1])]]
            set_col(u, fan[j + 1], -1)
            set_col(u, fan[j], cj)
        set_col(u, fan[widx], dcol)
    assert np.all(colour >= 0)
    return colour.astype(np.int32)


def check_colouring(n: int, edges: np.ndarray, colour: np.ndarray) -> bool:
    """True iff every colour class is a matching (no shared endpoints)."""
    seen = set()
    for (u, v), c in zip(np.asarray(edges).tolist(), np.asarray(colour).tolist()):
        if c < 0:
            return False
        for x in (u, v):
            if (x, c) in seen:
                return False
            seen.add((x, c))
    return True


@dataclasses.dataclass
class Instance:
    """One annealing problem: graph, couplings, fields and gate schedule."""
    n: int
    edges: np.ndarray    # (m, 2) int32, u < v, sorted
    J: np.ndarray        # (m,) float64
    h: np.ndarray        # (n,) float64
    colour: np.ndarray   # (m,) int32 proper edge colouring
    seed: int
    kind: str = "regular"

    @property
    def m(self) -> int:
        return int(self.edges.shape[0])

    @property
    def n_colours(self) -> int:
        return int(self.colour.max()) + 1 if self.m else 0


def make_instance(n: int, seed: int, d: int = 3, J: str = "gauss", h_std: float = 0.1,
                  base: int = BASE_SEED) -> Instance:
    """Random d-regular instance.  Graph seed base+3s, J seed base+3s+1, h seed base+3s+2.

    J: "gauss" (N(0,1)), "ferro" (+1 on all edges) or "maxcut" (-1 on all edges).
    h_std: standard deviation of the Gaussian fields (0 gives h = 0).
    """
    s = base + 3 * int(seed)
    edges = random_regular_graph(n, d, s)
    m = edges.shape[0]
    if J == "gauss":
        Jv = _rng(s + 1).normal(0.0, 1.0, size=m)
    elif J == "ferro":
        Jv = np.ones(m)
    elif J == "maxcut":
        Jv = -np.ones(m)
    else:
        raise ValueError(J)
    hv = _rng(s + 2).normal(0.0, h_std, size=n) if h_std > 0 else np.zeros(n)
    colour = edge_colouring(n, edges)
    return Instance(n, edges, Jv.astype(np.float64), hv.astype(np.float64), colour, int(seed))


def make_tree_instance(n: int, seed: int, h_std: float = 0.1, base: int = BASE_SEED,
                       max_degree: int = 3) -> Instance:
    """Random tree (max degree 3, or max_degree) with Gaussian J ~ N(0,1), h ~ N(0, h_std)."""
    s = base + 1_000_000 + 3 * int(seed) + (0 if max_degree == 3 else 100_000 * max_degree)
    edges = random_tree(n, s, max_degree)
    m = edges.shape[0]
    Jv = _rng(s + 1).normal(0.0, 1.0, size=m)
    hv = _rng(s + 2).normal(0.0, h_std, size=n) if h_std > 0 else np.zeros(n)
    colour = edge_colouring(n, edges)
    return Instance(n, edges, Jv, hv, colour, int(seed), kind="tree")


def make_heavy_hex_instance(rows: int, cols: int, seed: int, h_std: float = 0.1,
                            base: int = BASE_SEED) -> Instance:
    """Heavy-hexagon lattice with Gaussian J ~ N(0,1), h ~ N(0, h_std)."""
    s = base + 2_000_000 + 3 * int(seed)
    n, edges = heavy_hex_graph(rows, cols)
    m = edges.shape[0]
    Jv = _rng(s + 1).normal(0.0, 1.0, size=m)
    hv = _rng(s + 2).normal(0.0, h_std, size=n) if h_std > 0 else np.zeros(n)
    colour = edge_colouring(n, edges)
    return Instance(n, edges, Jv, hv, colour, int(seed), kind="heavy_hex")


def make_batch(B: int, seed: int = 0, n_lo: int = 50, n_hi: int = 1000) -> List[Instance]:
    """B random 3-regular instances with n uniform over even values in [n_lo, n_hi]."""
    rng = _rng(BASE_SEED + 7_000_000 + int(seed))
    ns = 2 * rng.integers(n_lo // 2, n_hi // 2 + 1, size=B)
    return [make_instance(int(ns[b]), seed=10_000 + 1000 * int(seed) + b) for b in range(B)]


def random_messages_input(shape, seed: int) -> np.ndarray:
    """Seeded i.i.d. complex normal matrices (re, im ~ N(0,1)), for random BP starts."""
    rng = _rng(seed)
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def random_gate_inputs(n: int, m: int, k2: int, k1: int, seed: int):
    """Seeded inputs for arbitrary-gate circuits: k2 two-qubit gates on uniformly drawn
    edges (repeats allowed) and k1 one-qubit gates on uniformly drawn vertices, each a
    Haar-distributed unitary (QR of a complex Gaussian matrix, phases of R's diagonal
    divided out).  Returns (edge ids (k2,), U (k2, 4, 4), vertex ids (k1,), W (k1, 2, 2))."""
    rng = _rng(BASE_SEED + 5_000_000 + int(seed))

    def haar(d):
        A = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
        Q, R = np.linalg.qr(A)
        return Q * (np.diag(R) / np.abs(np.diag(R)))[None, :]

    e = rng.integers(0, m, size=k2).astype(np.int32)
    U = np.stack([haar(4) for _ in range(k2)]) if k2 else np.zeros((0, 4, 4), complex)
    v = rng.integers(0, n, size=k1).astype(np.int32)
    W = np.stack([haar(2) for _ in range(k1)]) if k1 else np.zeros((0, 2, 2), complex)
    return e, U, v, W
