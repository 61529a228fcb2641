"""Seeded instance generators: shape, simplicity, regularity, colouring validity."""
import numpy as np
import pytest

from instances import (check_colouring, edge_colouring, make_batch, make_instance,
                       make_tree_instance, random_regular_graph, random_tree)


@pytest.mark.parametrize("n,seed", [(16, 0), (16, 7), (100, 3), (1000, 0)])
def test_regular_graph_is_simple_and_regular(n, seed):
    e = random_regular_graph(n, 3, seed)
    assert e.shape == (3 * n // 2, 2)
    assert np.all(e[:, 0] < e[:, 1])
    assert len({tuple(x) for x in e.tolist()}) == e.shape[0]
    assert np.all(np.bincount(e.ravel(), minlength=n) == 3)


def test_regular_graph_matches_networkx_degree_view():
    nx = pytest.importorskip("networkx")
    e = random_regular_graph(50, 3, 11)
    g = nx.Graph()
    g.add_edges_from(e.tolist())
    assert nx.is_regular(g) and all(d == 3 for _, d in g.degree())
    assert g.number_of_edges() == 75


def test_seeded_determinism():
    a, b = make_instance(40, 5), make_instance(40, 5)
    assert np.array_equal(a.edges, b.edges) and np.array_equal(a.J, b.J) and np.array_equal(a.h, b.h)
    c = make_instance(40, 6)
    assert not np.array_equal(a.J, c.J)


@pytest.mark.parametrize("seed", range(20))
def test_colouring_is_proper_with_at_most_four_colours(seed):
    inst = make_instance(16 + 2 * seed, seed)
    assert check_colouring(inst.n, inst.edges, inst.colour)
    assert inst.n_colours <= 4
    t = make_tree_instance(16, seed)
    assert check_colouring(t.n, t.edges, t.colour) and t.n_colours <= 4


def test_colouring_large_graph():
    inst = make_instance(1000, 0)
    assert check_colouring(inst.n, inst.edges, inst.colour) and inst.n_colours <= 4
    sizes = np.bincount(inst.colour)
    assert sizes.sum() == 1500 and sizes.max() <= 500


def test_check_colouring_rejects_shared_vertex():
    e = np.array([[0, 1], [1, 2]])
    assert not check_colouring(3, e, np.array([0, 0]))
    assert check_colouring(3, e, np.array([0, 1]))


def test_tree_has_max_degree_three():
    e = random_tree(30, 4)
    assert e.shape == (29, 2)
    assert np.bincount(e.ravel(), minlength=30).max() <= 3


def test_batch_sizes_even_in_range():
    b = make_batch(8, seed=0)
    assert len(b) == 8
    assert all(50 <= x.n <= 1000 and x.n % 2 == 0 for x in b)


@pytest.mark.parametrize("rows,cols", [(3, 9), (7, 15), (12, 27)])
def test_heavy_hex_lattice_structure(rows, cols):
    """Degree <= 3, connected, bipartite (all cycles even), shortest cycle 12."""
    from instances import heavy_hex_graph
    n, edges = heavy_hex_graph(rows, cols)
    deg = np.bincount(edges.ravel(), minlength=n)
    assert deg.max() <= 3 and deg.min() >= 1
    adj = [[] for _ in range(n)]
    for u, v in edges.tolist():
        adj[u].append(v)
        adj[v].append(u)
    colour = -np.ones(n, dtype=int)
    colour[0] = 0
    queue = [0]
    while queue:
        u = queue.pop()
        for v in adj[u]:
            if colour[v] < 0:
                colour[v] = 1 - colour[u]
                queue.append(v)
            assert colour[v] != colour[u]
    assert (colour >= 0).all()
    # girth by BFS from every vertex
    girth = np.inf
    for s in range(n):
        dist = {s: 0}
        parent = {s: -1}
        q = [s]
        for u in q:
            for v in adj[u]:
                if v not in dist:
                    dist[v] = dist[u] + 1
                    parent[v] = u
                    q.append(v)
                elif parent[u] != v:
                    girth = min(girth, dist[u] + dist[v] + 1)
    assert girth == 12
    c = edge_colouring(n, edges)
    assert check_colouring(n, edges, c)


def test_random_gate_inputs_are_unitary_and_seeded():
    from instances import random_gate_inputs
    e, U, v, W = random_gate_inputs(10, 12, 20, 7, seed=3)
    assert e.min() >= 0 and e.max() < 12 and v.min() >= 0 and v.max() < 10
    assert np.abs(U @ np.conj(np.swapaxes(U, 1, 2)) - np.eye(4)).max() < 1e-12
    assert np.abs(W @ np.conj(np.swapaxes(W, 1, 2)) - np.eye(2)).max() < 1e-12
    e2, U2, _, _ = random_gate_inputs(10, 12, 20, 7, seed=3)
    assert np.array_equal(e, e2) and np.array_equal(U, U2)


@pytest.mark.parametrize("seed", range(4))
def test_delta_colouring_of_cubic_graphs_trees_and_heavy_hex(seed):
    """The Kempe-chain search finds Delta = 3 colours on random cubic graphs (n = 1000),
    trees and heavy-hex lattices, and the result is a proper colouring."""
    from instances import delta_edge_colouring, make_heavy_hex_instance
    for inst in (make_instance(1000, seed), make_tree_instance(40, seed), make_heavy_hex_instance(4, 11, seed)):
        assert check_colouring(inst.n, inst.edges, inst.colour)
        assert inst.n_colours == 3
        col = delta_edge_colouring(inst.n, inst.edges, seed=seed + 1)
        assert col is not None and check_colouring(inst.n, inst.edges, col) and col.max() == 2


def test_delta_colouring_gives_up_on_the_petersen_graph():
    """The Petersen graph is cubic but needs 4 colours: the search gives up and edge_colouring
    falls back to Misra-Gries."""
    from instances import delta_edge_colouring
    outer = [(i, (i + 1) % 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    edges = np.array(sorted((min(a, b), max(a, b)) for a, b in outer + inner + spokes), dtype=np.int32)
    assert delta_edge_colouring(10, edges, max_steps=3000) is None
    col = edge_colouring(10, edges)
    assert check_colouring(10, edges, col) and col.max() == 3
