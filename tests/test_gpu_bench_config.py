"""GPU parity in the launch configuration the bench times, at the full size of the single-
instance workload (random 3-regular n = 1000, chi = 4, K = 3200, dt = 0.2, BP tol 1e-8, at most
100 sweeps): one-layer CUDA-graph replays (gtqa_anneal_graph) with the launch shapes that
gtqa_autotune picks for this workload (mixed: gates in 256-thread blocks, the regauge in
512-thread blocks with 64-thread vertex teams; FP64: the default shapes).

The first layers are compared with the oracle's own anneal.  In the late anneal, where BP stops
at max_iter, the oracle cannot follow the whole run; there one further flooding sweep is
checked message by message on sampled vertices against the oracle's update (Eq.
(local_consistency), normalised by the complex trace) of the device's incoming messages."""
import numpy as np
import pytest

import gpu_util as U
from instances import make_instance
from oracle import gtqa_oracle as O

pytestmark = pytest.mark.gpu
K, DT, TOL, MI, CHI = 3200, 0.2, 1e-8, 100, 4
SHAPES = {0: (0, 0, 0), 1: (1, 0, 2)}   # FP64, mixed: (gates, BP, regauge) variants


@pytest.fixture(scope="module")
def first_layers():
    inst = make_instance(1000, 0)
    st = O.plus_state(inst.n, inst.edges)
    for k in range(1, 4):
        tZ, tX = O.schedule(k, K, DT)
        st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, CHI, TOL, MI)
    return inst, st, O.reduced_density_matrices(st)


def _state(G, inst, prec):
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, CHI, inst.colour, G.gtqa_options_init(precision=prec))
    G.gtqa_set_shape(s, SHAPES[prec])
    return s


@pytest.mark.parametrize("prec, tol", [(0, 1e-9), (1, 1e-4)])
def test_first_layers_in_the_bench_configuration_match_the_oracle(first_layers, prec, tol):
    """Layers 1..3 through the graph with the tuned shapes: marginals and lambda against the
    oracle (1e-9 in FP64 as for the direct launches, 1e-4 in the mixed mode), and identical
    signs on every vertex clear of the read-out tie."""
    G = U.lib()
    inst, st, rho_o = first_layers
    s = _state(G, inst, prec)
    try:
        G.gtqa_anneal_graph(s, 1, 3, K, DT, TOL, MI)
        rho, sign = G.gtqa_marginals(s)
        _, L, _ = G.gtqa_get_state(s)
    finally:
        G.gtqa_destroy(s)
    assert np.abs(rho - rho_o).max() < tol, np.abs(rho - rho_o).max()
    _, Lo = O.to_padded(st, L.shape[1])
    assert np.abs(L - Lo).max() < tol, np.abs(L - Lo).max()
    clear = np.abs(rho_o[:, 0, 0].real - 0.5) > 1e-3
    sign_o = np.where(rho_o[:, 0, 0].real > 0.5, 1, -1)
    assert np.array_equal(np.asarray(sign)[clear], sign_o[clear])   # none may be clear this early


@pytest.mark.parametrize("prec, tol", [(0, 1e-11), (1, 2e-5)])
def test_late_anneal_sweep_in_the_bench_configuration_matches_the_oracle_update(prec, tol):
    """After layers 1..1500 through the graph with the tuned shapes (BP at max_iter in the
    last layers), one more flooding sweep without the warm start: on 24 sampled vertices every
    outgoing message equals the oracle's normalised update of the incoming messages before the
    sweep, with T the symmetric gauge of the device's Gamma and lambda (1e-11 in FP64; 2e-5 in
    the mixed mode, whose contractions run in FP32)."""
    G = U.lib()
    inst = make_instance(1000, 0)
    s = _state(G, inst, prec)
    try:
        G.gtqa_anneal_graph(s, 1, 1500, K, DT, TOL, MI)
        assert G.gtqa_stats(s)["bp_not_converged_calls"] > 0
        Gg, Lg, M0 = G.gtqa_get_state(s)
        G.gtqa_bp_sweep(s, 0.0, 1, 0)   # one sweep from the current messages, no regauge
        _, _, M1 = G.gtqa_get_state(s)
    finally:
        G.gtqa_destroy(s)
    inc = O.incidence(inst.n, inst.edges)
    rng = np.random.default_rng(7)
    worst = 0.0
    for a in rng.choice(inst.n, size=24, replace=False):
        a = int(a)
        st, msgs = U.star_state(Gg, Lg, M0, inst.edges, inc, a)
        T = O.symmetric_gauge(st)
        for q, e in enumerate(inc[a]):
            upd = O.message_update(st, T, msgs, 0, q)
            upd = upd / np.trace(upd)
            out = 2 * e + (0 if inst.edges[e][0] == a else 1)
            d = st.lam[q].size
            worst = max(worst, float(np.abs(upd - M1[out, :d, :d]).max()))
    assert worst < tol, worst
