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
