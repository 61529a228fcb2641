"""The C-ABI library loads on a machine without a GPU, exports every declared
entry point, and rejects invalid arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from instances import check_colouring, edge_colouring, make_instance, random_regular_graph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def G():
    from paper_2409_12240_gb300 import gtqa
    gtqa.load(build_if_missing=True)
    return gtqa


def _declared():
    src = open(os.path.join(ROOT, "include", "gtqa.h")).read()
    return sorted(set(re.findall(r"\b(gtqa_[a-z_0-9]+)\s*\(", src)))


def test_header_declarations_are_exported(G):
    lib = ctypes.CDLL(G.library_path())
    names = _declared()
    assert len(names) >= 14
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(names) == set(G.EXPORTED)


def test_strerror_codes(G):
    for c in range(8):
        assert len(G.strerror(c)) > 0
    assert G.strerror(99) == "unknown error code"


def test_options_init_selects_the_precision_default_cutoffs(G):
    """The initialiser leaves both cut-offs at 0, which gtqa_create reads as the precision's own
    default (1e-14 / 1e-13, or 1e-7 / 1e-6 in the complex64 mode); writing the FP64 values there
    made complex64 states keep FP32-noise singular values."""
    o = G.gtqa_options()
    G.load().gtqa_options_init(ctypes.byref(o))
    assert o.precision == G.GTQA_FP64 and o.svd_cutoff == 0.0 and o.eig_cutoff == 0.0
    assert o.cuda_stream is None
    o2 = G.gtqa_options_init(precision=G.GTQA_C64, svd_cutoff=1e-6)
    assert o2.precision == G.GTQA_C64 and o2.svd_cutoff == 1e-6 and o2.eig_cutoff == 0.0


@pytest.mark.parametrize("n,seed", [(16, 0), (50, 1), (1000, 2)])
def test_library_colouring_is_proper(G, n, seed):
    e = random_regular_graph(n, 3, seed)
    col, k = G.gtqa_edge_colouring(n, e)
    assert k <= 4 and check_colouring(n, e, col)


def _rc(G, n, edges, J, h, chi, colour=None, precision=0):
    opt = G.gtqa_options_init(precision=precision)
    handle = ctypes.c_void_p()
    edges = np.ascontiguousarray(edges, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    col = None if colour is None else np.ascontiguousarray(colour, dtype=np.int32)
    rc = G.load().gtqa_create(n, edges.shape[0], edges.ctypes.data, None if col is None else col.ctypes.data,
                              J.ctypes.data, h.ctypes.data, chi, ctypes.byref(opt), ctypes.byref(handle))
    return rc, handle.value


def test_invalid_graphs_rejected_on_host(G):
    h = np.zeros(4)
    # self-loop
    assert _rc(G, 4, [[0, 0]], [1.0], h, 4)[0] == G.GTQA_ERR_INVALID_ARG
    # duplicate edge
    assert _rc(G, 4, [[0, 1], [1, 0]], [1.0, 1.0], h, 4)[0] == G.GTQA_ERR_INVALID_ARG
    # degree 5
    star = [[0, 1], [0, 2], [0, 3], [0, 4], [0, 5]]
    assert _rc(G, 6, star, np.ones(5), np.zeros(6), 4)[0] == G.GTQA_ERR_INVALID_ARG
    # degree 4 needs chi <= 4 in every precision (checked before any device work)
    star4 = star[:4]
    for prec in (G.GTQA_FP64, G.GTQA_MIXED, G.GTQA_C64):
        assert _rc(G, 5, star4, np.ones(4), np.zeros(5), 8, precision=prec)[0] == G.GTQA_ERR_UNSUPPORTED
    # chi 9..16 (storage 16) needs degree <= 3
    assert _rc(G, 5, star4, np.ones(4), np.zeros(5), 12)[0] == G.GTQA_ERR_UNSUPPORTED
    assert _rc(G, 4, [[0, 1]], [1.0], h, 17)[0] == G.GTQA_ERR_UNSUPPORTED
    # out of range vertex
    assert _rc(G, 4, [[0, 7]], [1.0], h, 4)[0] == G.GTQA_ERR_INVALID_ARG
    # colouring that is not a matching
    assert _rc(G, 4, [[0, 1], [1, 2]], [1.0, 1.0], h, 4, colour=[0, 0])[0] == G.GTQA_ERR_INVALID_ARG
    # NaN coupling
    assert _rc(G, 4, [[0, 1]], [np.nan], h, 4)[0] == G.GTQA_ERR_INVALID_ARG
    # unsupported bond dimension / precision
    assert _rc(G, 4, [[0, 1]], [1.0], h, 64)[0] == G.GTQA_ERR_UNSUPPORTED
    assert _rc(G, 4, [[0, 1]], [1.0], h, 0)[0] == G.GTQA_ERR_INVALID_ARG


def test_null_handles_are_rejected(G):
    lib = G.load()
    assert lib.gtqa_trotter_layer(None, 0.5, 0.1) == G.GTQA_ERR_INVALID_ARG
    assert lib.gtqa_regauge(None) == G.GTQA_ERR_INVALID_ARG
    three = (ctypes.c_int32 * 3)(0, 0, 0)
    table = (ctypes.c_int32 * 12)()
    assert lib.gtqa_set_shape(None, three) == G.GTQA_ERR_INVALID_ARG
    assert lib.gtqa_launch_shape(None, table) == G.GTQA_ERR_INVALID_ARG
    lib.gtqa_destroy(None)


def test_set_shape_wants_one_variant_per_phase_kernel(G):
    """The binding checks the shape of the variant list before it reaches the library."""
    for bad in ((0, 0), (0, 0, 0, 0), ((0, 0, 0),)):
        with pytest.raises(ValueError):
            G.gtqa_set_shape(0, bad)


def test_library_colouring_uses_delta_colours_when_it_can(G):
    """Random cubic graphs (n up to 100000), trees and heavy-hex lattices get 3 colours; the
    Petersen graph and a cubic graph with a bridge (both class 2) fall back to Misra-Gries
    with 4."""
    from instances import heavy_hex_graph, random_tree
    for n, seed in ((50, 1), (1000, 3), (100000, 2)):
        e = random_regular_graph(n, 3, seed)
        col, k = G.gtqa_edge_colouring(n, e)
        assert k == 3 and check_colouring(n, e, col)
    e = random_regular_graph(16, 3, 0)     # has the bridge {4, 5}
    col, k = G.gtqa_edge_colouring(16, e)
    assert k == 4 and check_colouring(16, e, col)
    t = random_tree(60, 4)
    col, k = G.gtqa_edge_colouring(60, t)
    assert k == 3 and check_colouring(60, t, col)
    nh, eh = heavy_hex_graph(7, 15)
    col, k = G.gtqa_edge_colouring(nh, eh)
    assert k == 3 and check_colouring(nh, eh, col)
    outer = [(i, (i + 1) % 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    pe = np.array(sorted((min(a, b), max(a, b)) for a, b in outer + inner + spokes), dtype=np.int32)
    col, k = G.gtqa_edge_colouring(10, pe)
    assert k == 4 and check_colouring(10, pe, col)


def test_gate_layering_keeps_order_and_disjointness(G):
    """gtqa_apply_gates' launch layering: gates of one launch have disjoint endpoints, two gates
    sharing a vertex keep their list order, and each gate sits one launch after its latest
    predecessor on a shared vertex (so the layering is as shallow as the order allows)."""
    from instances import random_gate_inputs
    n = 40
    e = random_regular_graph(n, 3, 4)
    gate_e, _, _, _ = random_gate_inputs(n, e.shape[0], 400, 0, seed=9)
    lay, nl = G.gtqa_gate_layers(n, e, gate_e)
    assert nl == lay.max() + 1
    depth = np.zeros(n, dtype=int)
    for q, ed in enumerate(gate_e.tolist()):
        a, b = e[ed]
        assert lay[q] == max(depth[a], depth[b])
        depth[a] = depth[b] = lay[q] + 1
    for L in range(nl):
        verts = e[gate_e[lay == L]].ravel()
        assert np.unique(verts).size == verts.size
    # one colour class of a proper colouring is a single launch
    col = edge_colouring(n, e)
    lay1, nl1 = G.gtqa_gate_layers(n, e, np.nonzero(col == 0)[0])
    assert nl1 == 1 and (lay1 == 0).all()
    with pytest.raises(Exception):
        G.gtqa_gate_layers(n, e, [e.shape[0]])
