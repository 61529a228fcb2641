"""The fused multi-layer launch, batching and the bounded-barrier failure path."""
import numpy as np
import pytest

import gpu_util as U
from instances import make_instance

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_fused_anneal_equals_stepwise_calls(precision):
    G = U.lib()
    inst = make_instance(40, 3)
    opt = G.gtqa_options_init(precision=precision)
    a = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour, opt)
    b = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour, opt)
    try:
        K, dt, tol, mi = 30, 0.2, 1e-9, 60
        G.gtqa_anneal(a, 1, 12, K, dt, tol, mi)
        G.gtqa_anneal(a, 13, 20, K, dt, tol, mi)
        for k in range(1, 21):
            G.gtqa_trotter_layer(b, k / K, dt)
            G.gtqa_bp_sweep(b, tol, mi)
        ra, _ = G.gtqa_marginals(a)
        rb, _ = G.gtqa_marginals(b)
        assert np.array_equal(ra, rb)
        Ga, La, _ = G.gtqa_get_state(a)
        Gb, Lb, _ = G.gtqa_get_state(b)
        assert np.array_equal(Ga, Gb) and np.array_equal(La, Lb)
        sa, sb = G.gtqa_stats(a), G.gtqa_stats(b)
        assert sa["bp_sweeps"] == sb["bp_sweeps"] and sa["layers"] == sb["layers"] == 20
        assert sa["bp_calls"] == 20
    finally:
        G.gtqa_destroy(a)
        G.gtqa_destroy(b)


def test_batch_per_instance_convergence_matches_single_runs():
    G = U.lib()
    insts = [make_instance(n, 40 + i) for i, n in enumerate((16, 30, 50, 24))]
    sb = G.gtqa_create_batch([x.n for x in insts], [x.edges for x in insts], [x.J for x in insts],
                             [x.h for x in insts], 4, [x.colour for x in insts])
    singles = [G.gtqa_create(x.n, x.edges, x.J, x.h, 4, x.colour) for x in insts]
    try:
        G.gtqa_anneal(sb, 1, 10, 20, 0.2, 1e-10, 80)
        for s in singles:
            G.gtqa_anneal(s, 1, 10, 20, 0.2, 1e-10, 80)
        rb, _ = G.gtqa_marginals(sb)
        rs = np.concatenate([G.gtqa_marginals(s)[0] for s in singles])
        assert np.abs(rb - rs).max() < 1e-12
    finally:
        G.gtqa_destroy(sb)
        for s in singles:
            G.gtqa_destroy(s)


def test_barrier_timeout_is_reported_and_context_survives():
    """A grid barrier that waits for a block that does not exist gives up after its poll
    budget; the library reports GTQA_ERR_TIMEOUT and the device stays usable."""
    G = U.lib()
    inst = make_instance(16, 0)
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour)
    try:
        G.gtqa_debug_barrier(s, 20000, 1)
        G.gtqa_trotter_layer(s, 0.5, 0.1)   # asynchronous; the failure shows at the next sync
        with pytest.raises(G.GTQAError) as ei:
            G.gtqa_bp_sweep(s, 1e-8, 10)
        assert ei.value.code == G.GTQA_ERR_TIMEOUT
        with pytest.raises(G.GTQAError):
            G.gtqa_trotter_layer(s, 0.5, 0.1)   # sticky
    finally:
        G.gtqa_destroy(s)
    s2 = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour)
    try:
        G.gtqa_trotter_layer(s2, 0.5, 0.1)
        it, d, conv = G.gtqa_bp_sweep(s2, 1e-10, 100)
        assert conv
    finally:
        G.gtqa_destroy(s2)


def test_newton_refined_reciprocal_and_roots_match_cuda():
    """The kernels replace FP64 divide/sqrt by Newton-Raphson refinement of the PTX
    approximations; they must agree with CUDA's correctly rounded results to a few ulp."""
    G = U.lib()
    rng = np.random.default_rng(0)
    x = np.concatenate([10.0 ** rng.uniform(-250, 250, 4000), rng.uniform(0.5, 2.0, 1000), [1.0, 2.0, 4.0, 1e-30]])
    out = G.gtqa_math_check(x)
    for a, b in ((0, 1), (2, 3), (4, 5)):
        rel = np.abs(out[:, a] - out[:, b]) / np.abs(out[:, b])
        assert rel.max() < 4 * np.finfo(float).eps, (a, rel.max())


@pytest.mark.parametrize("precision", [0, 1])
def test_anneal_from_a_cuda_graph_matches_direct_launches(precision):
    """gtqa_anneal_graph (layers captured once into a CUDA graph) gives the state of gtqa_anneal,
    bit for bit, for a first range, a replay of a new range, and a batched state."""
    import numpy as np
    from instances import make_batch, make_instance
    G = U.lib()
    K, dt, tol, mi = 200, 0.2, 1e-8, 100
    for kind in ("single", "batch"):
        out = []
        for graph in (False, True):
            opt = G.gtqa_options_init(precision=precision)
            if kind == "single":
                inst = make_instance(200, 5)
                s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour, opt)
            else:
                insts = make_batch(6, seed=3, n_lo=50, n_hi=120)
                s = G.gtqa_create_batch([x.n for x in insts], [x.edges for x in insts], [x.J for x in insts],
                                        [x.h for x in insts], 4, [x.colour for x in insts], opt)
            try:
                for k0, k1 in ((1, 8), (9, 20)):
                    if graph:
                        G.gtqa_anneal_graph(s, k0, k1, K, dt, tol, mi)
                    else:
                        G.gtqa_anneal(s, k0, k1, K, dt, tol, mi)
                out.append((G.gtqa_get_state(s), G.gtqa_marginals(s)[0], G.gtqa_stats(s)))
            finally:
                G.gtqa_destroy(s)
        (sa, ra, ta), (sb, rb, tb) = out
        for a, b in zip(sa, sb):
            assert np.array_equal(a, b), kind
        assert np.array_equal(ra, rb)
        assert ta["layers"] == tb["layers"] == 20 and ta["bp_calls"] == tb["bp_calls"] == 20


def test_profiled_graph_replays_time_each_phase_and_keep_results():
    """With the profiler on, every graph replay is timed into the gates, BP and regauge classes
    (one launch of each per layer) and the state stays that of direct launches, bit for bit."""
    import numpy as np
    from instances import make_instance
    G = U.lib()
    inst = make_instance(200, 6)
    K, dt, tol, mi = 200, 0.2, 1e-8, 100
    out = []
    for graph in (False, True):
        s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour, G.gtqa_options_init(precision=1))
        try:
            G.gtqa_anneal(s, 1, 5, K, dt, tol, mi)
            G.gtqa_profile(s, True)
            if graph:
                G.gtqa_anneal_graph(s, 6, 17, K, dt, tol, mi)
            else:
                G.gtqa_anneal(s, 6, 17, K, dt, tol, mi)
            prof = G.gtqa_profile_read(s)
            G.gtqa_profile(s, False)
            G.gtqa_anneal_graph(s, 18, 20, K, dt, tol, mi) if graph else G.gtqa_anneal(s, 18, 20, K, dt, tol, mi)
            out.append((G.gtqa_get_state(s), prof))
        finally:
            G.gtqa_destroy(s)
    (sa, pa), (sb, pb) = out
    for a, b in zip(sa, sb):
        assert np.array_equal(a, b)
    for name in ("gates_kernel", "bp_kernel", "regauge_kernel"):
        assert pa[name][0] == pb[name][0] == 12, (name, pa[name], pb[name])
        assert pb[name][1] > 0.0 and pa[name][2] == pb[name][2]
        # the same device work, timed by events around the launches or between graph nodes
        assert 0.5 < pb[name][1] / pa[name][1] < 2.0, (name, pa[name], pb[name])


def test_autotune_restores_the_state_and_keeps_results():
    """gtqa_autotune leaves the state and statistics as they were, keeps grid sizes within the SM
    count, and the layers it then runs give the results of the default launch shapes (FP64; a
    different BP vertex team changes only the rounding order of its sums)."""
    import numpy as np
    from instances import make_instance
    G = U.lib()
    inst = make_instance(1000, 0)
    K, dt, tol, mi = 3200, 0.2, 1e-10, 100
    res = []
    for tune in (False, True):
        s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour, G.gtqa_options_init(precision=0))
        try:
            G.gtqa_anneal(s, 1, 30, K, dt, tol, mi)
            before = G.gtqa_get_state(s)
            st0 = G.gtqa_stats(s)
            if tune:
                grid = G.gtqa_autotune(s, 31 / K, dt, tol, mi)
                assert all(1 <= g <= 152 for g in grid), grid
                after = G.gtqa_get_state(s)
                for a, b in zip(before, after):
                    assert np.array_equal(a, b)
                st1 = G.gtqa_stats(s)
                for k in ("layers", "gates", "bp_calls", "bp_sweeps", "discarded_weight"):
                    assert st0[k] == st1[k], k
            G.gtqa_anneal(s, 31, 40, K, dt, tol, mi)
            res.append((G.gtqa_get_state(s)[1], G.gtqa_marginals(s)[0]))
        finally:
            G.gtqa_destroy(s)
    assert np.abs(res[0][0] - res[1][0]).max() < 1e-12 and np.abs(res[0][1] - res[1][1]).max() < 1e-12
