"""Launch-shape variants of the persistent phase kernels (threads per block, BP vertex team,
regauge-vertex team) and the autotuner's search over them.

Every variant computes the same layer (simple update and truncation of Sec. II B / App. E,
flooding BP with the stopping rule of App. B, Vidal gauge finding of App. C), so each one is
held to the oracle like the default shape: 1e-10 in FP64, 1e-4 on the marginals in the mixed
mode with the same sign read-out.  Across variants the results differ only in the rounding
order of BP's contraction sums (the BP vertex team splits the (i, u) sum over a different
number of lanes)."""
import numpy as np
import pytest

import gpu_util as U
from instances import make_instance
from oracle import gtqa_oracle as O

pytestmark = pytest.mark.gpu

# (gates, BP, regauge) variant triples: the default, every non-default variant at least once
SHAPES = [(0, 0, 0), (1, 1, 1), (0, 2, 2), (1, 2, 1)]


def _fp64(out, tol=1e-10):
    assert max(out["rho"]) < tol, out["rho"]
    assert max(out["lam"]) < tol, out["lam"]
    assert max(out["msg_abs"]) < tol, out["msg_abs"]
    assert max(out["gamma"]) < 1e-8, out["gamma"]


def _mixed(out):
    assert max(out["rho"]) < 1e-4, out["rho"]
    rho_g, sign_g = out["rho_gpu"]
    rho_o = O.reduced_density_matrices(out["state"])
    clear = np.abs(rho_o[:, 0, 0].real - 0.5) > 1e-3
    assert np.array_equal(sign_g[clear], O.rounding(rho_o)[clear])


def _fits(G, chi, precision, shape):
    """The FP64 BP kernel at CHI = 8 in 512-thread blocks with two 256-thread vertex teams needs
    more shared memory than an SM has (two FP64 caches of 2 CHI^3 tensors and their products)."""
    return not (chi == 8 and precision == G.GTQA_FP64 and shape[1] == 1)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("chi", [4, 8])
def test_every_shape_matches_the_oracle_fp64(chi, shape):
    G = U.lib()
    inst = make_instance(16, 5)
    if not _fits(G, chi, G.GTQA_FP64, shape):
        pytest.skip("variant does not fit on an SM (checked by test_a_shape_that_does_not_fit_is_refused)")
    out = U.run_pair(inst, chi, 20, 0.1, 1e-12, 100, 8, precision=G.GTQA_FP64, shape=shape)
    table = out["launch"]
    assert [table[k]["variant"] for k in ("gates_kernel", "bp_kernel", "regauge_kernel")] == list(shape)
    _fp64(out)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("chi", [4, 8])
def test_every_shape_matches_the_oracle_mixed(chi, shape):
    G = U.lib()
    inst = make_instance(16, 6)
    out = U.run_pair(inst, chi, 20, 0.1, 1e-12, 100, 8, precision=G.GTQA_MIXED, shape=shape)
    _mixed(out)


def test_launch_table_lists_threads_and_teams():
    """The launch table reports the compiled shapes: CHI = 4 gate teams of 2 CHI^2 = 32 threads,
    BP vertex teams of 64 or 128 threads, regauge-vertex teams of 32 or 64 threads."""
    G = U.lib()
    inst = make_instance(16, 1)
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour)
    try:
        t = G.gtqa_launch_shape(s)
        assert t["gates_kernel"] == {"grid": t["gates_kernel"]["grid"], "variant": 0, "threads_per_block": 512,
                                     "team": 32}
        assert (t["bp_kernel"]["threads_per_block"], t["bp_kernel"]["team"]) == (512, 64)
        assert (t["regauge_kernel"]["threads_per_block"], t["regauge_kernel"]["team"]) == (512, 32)
        G.gtqa_set_shape(s, (1, 2, 2))
        t = G.gtqa_launch_shape(s)
        assert (t["gates_kernel"]["threads_per_block"], t["gates_kernel"]["team"]) == (256, 32)
        assert (t["bp_kernel"]["threads_per_block"], t["bp_kernel"]["team"]) == (512, 128)
        assert (t["regauge_kernel"]["threads_per_block"], t["regauge_kernel"]["team"]) == (512, 64)
    finally:
        G.gtqa_destroy(s)


def test_a_shape_that_does_not_fit_is_refused():
    """Out-of-range indices are invalid arguments; a variant whose shared memory exceeds an SM's
    is refused with GTQA_ERR_UNSUPPORTED and the state keeps its shapes and keeps working."""
    G = U.lib()
    inst = make_instance(16, 2)
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 8, inst.colour)
    try:
        before = G.gtqa_launch_shape(s)
        for bad in ((2, 0, 0), (0, 3, 0), (0, 0, -1)):
            with pytest.raises(G.GTQAError) as ei:
                G.gtqa_set_shape(s, bad)
            assert ei.value.code == G.GTQA_ERR_INVALID_ARG
        with pytest.raises(G.GTQAError) as ei:
            G.gtqa_set_shape(s, (1, 1, 1))
        assert ei.value.code == G.GTQA_ERR_UNSUPPORTED
        assert G.gtqa_launch_shape(s) == before
        G.gtqa_trotter_layer(s, 0.05, 0.1)
        it, dist, conv = G.gtqa_bp_sweep(s, 1e-10, 50)
        assert conv
    finally:
        G.gtqa_destroy(s)


def test_graph_replays_follow_a_new_shape():
    """A layer graph captured before gtqa_set_shape is dropped: replays after the change run the
    new shapes and give the results of direct launches with those shapes."""
    G = U.lib()
    inst = make_instance(1000, 0)
    K, dt, tol, mi = 3200, 0.2, 1e-8, 100
    res = []
    for graph in (False, True):
        s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour, G.gtqa_options_init(precision=1))
        try:
            if graph:
                G.gtqa_anneal_graph(s, 1, 3, K, dt, tol, mi)
            else:
                G.gtqa_anneal(s, 1, 3, K, dt, tol, mi)
            G.gtqa_set_shape(s, (1, 2, 2))
            if graph:
                G.gtqa_anneal_graph(s, 4, 10, K, dt, tol, mi)
            else:
                G.gtqa_anneal(s, 4, 10, K, dt, tol, mi)
            res.append(G.gtqa_get_state(s))
        finally:
            G.gtqa_destroy(s)
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)


def test_autotune_picks_a_compiled_shape_and_keeps_results():
    """gtqa_autotune searches variants and grids; the table it leaves names compiled shapes, and
    the layers run with it stay within rounding of the default shapes (FP64, 1e-12)."""
    from instances import make_instance as mk
    G = U.lib()
    inst = mk(1000, 0)
    K, dt, tol, mi = 3200, 0.2, 1e-10, 100
    res, tables = [], []
    for tune in (False, True):
        s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour, G.gtqa_options_init(precision=0))
        try:
            G.gtqa_anneal(s, 1, 30, K, dt, tol, mi)
            if tune:
                G.gtqa_autotune(s, 31 / K, dt, tol, mi)
            tables.append(G.gtqa_launch_shape(s))
            G.gtqa_anneal(s, 31, 40, K, dt, tol, mi)
            res.append((G.gtqa_get_state(s)[1], G.gtqa_marginals(s)[0]))
        finally:
            G.gtqa_destroy(s)
    t = tables[1]
    assert 0 <= t["gates_kernel"]["variant"] <= 1
    assert 0 <= t["bp_kernel"]["variant"] <= 2 and 0 <= t["regauge_kernel"]["variant"] <= 2
    assert all(1 <= t[k]["grid"] <= 152 for k in t)
    assert np.abs(res[0][0] - res[1][0]).max() < 1e-12
    assert np.abs(res[0][1] - res[1][1]).max() < 1e-12
