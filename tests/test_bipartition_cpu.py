"""Host spectral bipartition of the library (Eq. (bipartition)) against the oracle's dense
computation: identical cuts where Lanczos spans the whole space (n <= 241) and the second
Laplacian eigenvalue is simple; a near-optimal split above."""
import numpy as np
import pytest

from instances import make_instance
from oracle import gtqa_oracle as O


@pytest.fixture(scope="module")
def G():
    from paper_2409_12240_gb300 import gtqa
    gtqa.load(build_if_missing=True)
    return gtqa


def _simple_lambda2(n, edges):
    L = np.zeros((n, n))
    for u, v in edges:
        L[u, v] -= 1
        L[v, u] -= 1
        L[u, u] += 1
        L[v, v] += 1
    w = np.linalg.eigvalsh(L)
    return w[2] - w[1] > 1e-6


def test_closed_forms(G):
    k4 = [(a, b) for a in range(4) for b in range(a + 1, 4)]
    edges = np.array(k4 + [(a + 4, b + 4) for a, b in k4] + [(3, 4)])
    side, cut, r = G.gtqa_spectral_bipartition(8, edges)
    assert abs(r - 1 / 16) < 1e-12 and cut.sum() == 1
    ring = np.array([(a, (a + 1) % 12) for a in range(12)])
    side, cut, r = G.gtqa_spectral_bipartition(12, ring)
    assert abs(r - 2 / 36) < 1e-12 and cut.sum() == 2


@pytest.mark.parametrize("n, seed", [(12, 0), (16, 1), (50, 2), (120, 3), (240, 4)])
def test_matches_oracle_in_the_exact_regime(G, n, seed):
    inst = make_instance(n, seed)
    if not _simple_lambda2(n, inst.edges):
        pytest.skip("degenerate second eigenvalue: the split is not unique")
    s_g, c_g, r_g = G.gtqa_spectral_bipartition(n, inst.edges)
    s_o, c_o, r_o = O.spectral_bipartition(n, inst.edges)
    assert abs(r_g - r_o) < 1e-12
    assert np.array_equal(c_g, c_o)
    assert np.array_equal(s_g, s_o) or np.array_equal(s_g, ~s_o)


def test_large_graph_is_consistent_and_near_the_dense_split(G):
    n = 1000
    inst = make_instance(n, 0)
    s_g, c_g, r_g = G.gtqa_spectral_bipartition(n, inst.edges)
    _, _, r_o = O.spectral_bipartition(n, inst.edges)
    e = inst.edges
    assert np.array_equal(c_g, s_g[e[:, 0]] != s_g[e[:, 1]])
    assert abs(r_g - c_g.sum() / (s_g.sum() * (n - s_g.sum()))) < 1e-15
    assert r_g < 1.2 * r_o


def test_rejects_bad_input(G):
    with pytest.raises(G.GTQAError):
        G.gtqa_spectral_bipartition(1, np.zeros((0, 2)))
    with pytest.raises(G.GTQAError):
        G.gtqa_spectral_bipartition(4, np.array([[0, 4]]))
