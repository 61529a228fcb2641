"""BP in the late anneal, where flooding BP stops at the maximal number of iterations
(App. B's exit at K iterations).

On the single-instance workload (n = 1000, h ~ N(0, 0.1)) BP reaches max_iter in every layer
from layer ~1230 on, far from converged.  Small instances of the same distribution reach it
much earlier, with a slowly falling distance: on n = 16, seed 6, K = 200, dt = 0.2, tol 1e-8
the oracle's BP needs more than 100 sweeps from layer 107 on.  The oracle anneals that
instance itself, and its state is the common input of the n = 16 checks, so no input of the
oracle comes from the CUDA path.
"""
import numpy as np
import pytest

import gpu_util as U
from instances import make_instance
from oracle import gtqa_oracle as O

pytestmark = pytest.mark.gpu
K, DT, TOL, MI, CHI = 200, 0.2, 1e-8, 100, 4
LATE = 110   # layers the oracle anneals before the checked layer (BP at max_iter from 107)


@pytest.fixture(scope="module")
def late_state():
    """The oracle's state after LATE layers, then the gates of layer LATE + 1, with the sweep
    counts of the oracle's BP in every layer."""
    inst = make_instance(16, 6)
    st = O.plus_state(inst.n, inst.edges)
    sweeps = []
    for k in range(1, LATE + 1):
        tZ, tX = O.schedule(k, K, DT)
        st, info = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, CHI, TOL, MI)
        sweeps.append(info["bp_iters"])
    tZ, tX = O.schedule(LATE + 1, K, DT)
    O.trotter_layer(st, inst.colour, inst.J, inst.h, tZ, tX, CHI)
    return inst, st, sweeps


def _gpu_state(G, inst, st, precision):
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, CHI, inst.colour, G.gtqa_options_init(precision=precision))
    n, m, C, _ = G.gtqa_sizes(s)
    Gp, Lp = O.to_padded(st, C)
    G.gtqa_set_state(s, Gp, Lp, np.zeros((2 * m, C, C), dtype=np.complex128))
    return s


def test_the_oracle_reaches_max_iter_in_the_late_anneal(late_state):
    _, _, sweeps = late_state
    assert all(x == MI for x in sweeps[106:]), sweeps[100:]
    assert max(sweeps[:90]) < MI, sweeps[:90]


def test_150_late_anneal_sweeps_then_regauge_match_the_oracle(late_state):
    """150 flooding sweeps from the warm start at tol 0 (after 100 sweeps the distance is still
    above tol), then Vidal gauge finding and the marginals: FP64 messages, lambda and rho within
    1e-10 of the oracle, the mixed path's rho within 1e-4."""
    inst, st0, _ = late_state
    G = U.lib()
    st = st0.copy()
    T = O.symmetric_gauge(st)
    msgs, it_o, hist = O.bp(st, T, O.reconstructed_messages(st), 0.0, 150)
    assert it_o == 150 and hist[MI - 1] > TOL, hist[MI - 1]   # why the oracle's layers stop at max_iter
    new = O.vidal_gauge(st, T, msgs)
    rho_o = O.reduced_density_matrices(new)
    _, L_o = O.to_padded(new, 4)
    s64 = _gpu_state(G, inst, st0, G.GTQA_FP64)
    smx = _gpu_state(G, inst, st0, G.GTQA_MIXED)
    try:
        it, dist, conv = G.gtqa_bp_sweep(s64, 0.0, 150, G.GTQA_BP_WARM_START)
        assert it == 150 and not conv and abs(dist - hist[-1]) < 1e-10
        _, _, Mg = G.gtqa_get_state(s64)
        Mo = O.messages_to_padded(st, msgs, 4)
        assert np.abs(Mg - Mo).max() < 1e-10, np.abs(Mg - Mo).max()
        G.gtqa_regauge(s64)
        rho64, sign64 = G.gtqa_marginals(s64)
        _, L64, _ = G.gtqa_get_state(s64)
        assert np.abs(L64 - L_o).max() < 1e-10
        assert np.abs(rho64 - rho_o).max() < 1e-10
        assert np.array_equal(sign64, O.rounding(rho_o))
        it, dist_m, conv = G.gtqa_bp_sweep(smx, 0.0, 150, G.GTQA_BP_WARM_START)
        assert it == 150 and abs(dist_m - hist[-1]) < 1e-4 * max(1.0, hist[-1])
        G.gtqa_regauge(smx)
        rho_m, _ = G.gtqa_marginals(smx)
        assert np.abs(rho_m - rho_o).max() < 1e-4, np.abs(rho_m - rho_o).max()
    finally:
        G.gtqa_destroy(s64)
        G.gtqa_destroy(smx)


def test_late_anneal_bp_stops_at_max_iter_like_the_oracle(late_state):
    """tol 1e-8, max_iter 100: both sides run the 100 sweeps and report the same distance."""
    inst, st0, _ = late_state
    G = U.lib()
    st = st0.copy()
    T = O.symmetric_gauge(st)
    _, it_o, hist = O.bp(st, T, O.reconstructed_messages(st), TOL, MI)
    s = _gpu_state(G, inst, st0, G.GTQA_FP64)
    try:
        it, dist, conv = G.gtqa_bp_sweep(s, TOL, MI, G.GTQA_BP_WARM_START)
        assert it == it_o == MI and not conv
        assert abs(dist - hist[-1]) < 1e-10
        assert G.gtqa_stats(s)["not_converged"] == 1
    finally:
        G.gtqa_destroy(s)


def test_sweep_counts_and_exact_distance_passes_along_the_anneal():
    """Layers 1..30 of the same instance from identical oracle states: the GPU's BP stops after
    the same sweep as the oracle's in every layer (the exact trace-norm rule of App. B), and
    some of those stops were decided by a separate exact-distance pass (a lower bound that
    fell under the threshold)."""
    inst = make_instance(16, 6)
    G = U.lib()
    st = O.plus_state(inst.n, inst.edges)
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, CHI, inst.colour)
    try:
        n, m, C, _ = G.gtqa_sizes(s)
        passes0 = G.gtqa_stats(s)["bp_exact_passes"]
        for k in range(1, 31):
            tZ, tX = O.schedule(k, K, DT)
            O.trotter_layer(st, inst.colour, inst.J, inst.h, tZ, tX, CHI)
            Gp, Lp = O.to_padded(st, C)
            G.gtqa_set_state(s, Gp, Lp, np.zeros((2 * m, C, C), dtype=np.complex128))
            it, dist, conv = G.gtqa_bp_sweep(s, TOL, MI, G.GTQA_BP_WARM_START)
            T = O.symmetric_gauge(st)
            msgs, it_o, hist = O.bp(st, T, O.reconstructed_messages(st), TOL, MI)
            assert it == it_o, (k, it, it_o, hist[-3:])
            assert abs(dist - hist[-1]) < 1e-12, (k, dist, hist[-1])
            st = O.vidal_gauge(st, T, msgs)
        assert G.gtqa_stats(s)["bp_exact_passes"] > passes0
    finally:
        G.gtqa_destroy(s)


@pytest.mark.slow
def test_late_anneal_mixed_against_fp64_at_n1000():
    """The single-instance workload at layer 1501 (BP at max_iter there): from the FP64 path's
    state after the gates, 150 sweeps at tol 0 and the regauge in FP64 and in the mixed mode;
    the mixed marginals stay within 1e-4 of FP64 and the signs agree where they are clear.  (The
    FP64 path itself is held to the oracle by the n = 16 checks above.)"""
    G = U.lib()
    inst = make_instance(1000, 0)
    Kf, dtf = 3200, 0.2
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, CHI, inst.colour)
    try:
        G.gtqa_anneal_graph(s, 1, 1500, Kf, dtf, TOL, MI)
        G.gtqa_trotter_layer(s, 1501 / Kf, dtf)
        Gm, L, _ = G.gtqa_get_state(s)
    finally:
        G.gtqa_destroy(s)
    out = []
    for p in (G.GTQA_FP64, G.GTQA_MIXED):
        s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, CHI, inst.colour, G.gtqa_options_init(precision=p))
        try:
            G.gtqa_set_state(s, Gm, L, np.zeros((2 * inst.m, 4, 4), dtype=np.complex128))
            it, dist, conv = G.gtqa_bp_sweep(s, 0.0, 150, G.GTQA_BP_WARM_START)
            assert it == 150 and dist > 1e-4   # far from converged
            G.gtqa_regauge(s)
            out.append((dist, G.gtqa_marginals(s)))
        finally:
            G.gtqa_destroy(s)
    (d64, (r64, s64)), (dmx, (rmx, smx)) = out
    assert abs(d64 - dmx) < 1e-3 * d64
    assert np.abs(r64 - rmx).max() < 1e-4, np.abs(r64 - rmx).max()
    clear = np.abs(r64[:, 0, 0].real - 0.5) > 1e-3
    assert np.array_equal(s64[clear], smx[clear])
