"""GPU FP64 path vs the CPU oracle, through the C ABI (parity bar: 1e-10 on
marginals, lambda and messages in FP64 mode)."""
import numpy as np
import pytest

import gpu_util as U
from instances import make_instance, make_tree_instance, Instance
from oracle import gtqa_oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _assert_parity(out, tol=TOL):
    assert max(out["rho"]) < tol, out["rho"]
    assert max(out["lam"]) < tol, out["lam"]
    assert max(out["msg_abs"]) < tol, out["msg_abs"]
    assert max(out["msg_spec"]) < tol, out["msg_spec"]
    assert max(out["gamma"]) < 1e-8, out["gamma"]


@pytest.mark.parametrize("seed", range(5))
def test_regular_n16_chi4_twenty_layers(seed):
    # 3-regular, n = 16, J ~ N(0,1), h ~ N(0, 0.1), 20 layers, dt = 0.1, chi = 4, tol 1e-12
    inst = make_instance(16, seed)
    out = U.run_pair(inst, 4, 20, 0.1, 1e-12, 100, 20)
    _assert_parity(out)
    assert all(abs(a - b) <= 1 for a, b in out["iters"]), out["iters"]


@pytest.mark.parametrize("chi", [1, 2, 3, 8])
def test_regular_n16_other_chi(chi):
    inst = make_instance(16, 7)
    out = U.run_pair(inst, chi, 20, 0.1, 1e-12, 100, 12)
    _assert_parity(out)


@pytest.mark.parametrize("seed", range(3))
def test_trees_with_phantom_slots(seed):
    inst = make_tree_instance(16, seed)
    out = U.run_pair(inst, 4, 20, 0.1, 1e-12, 100, 10)
    _assert_parity(out)


def test_two_qubits_single_edge():
    inst = Instance(2, np.array([[0, 1]], dtype=np.int32), np.array([0.8]), np.array([0.3, -0.2]),
                    np.zeros(1, dtype=np.int32), 0)
    out = U.run_pair(inst, 2, 10, 0.3, 1e-12, 100, 10)
    _assert_parity(out)


def test_zero_field_symmetry_and_product_state():
    inst = make_instance(16, 3, h_std=0.0)
    out = U.run_pair(inst, 4, 20, 0.1, 1e-12, 100, 8)
    _assert_parity(out)
    rho, _ = out["rho_gpu"]
    assert np.abs(rho[:, 0, 0].real - 0.5).max() < 1e-10
    inst = make_instance(16, 4)
    inst.J[:] = 0.0
    out = U.run_pair(inst, 4, 20, 0.1, 1e-12, 100, 6)
    _assert_parity(out)


def test_batch_matches_single_instances():
    G = U.lib()
    insts = [make_instance(n, 20 + i) for i, n in enumerate((16, 24, 40))]
    sb = G.gtqa_create_batch([x.n for x in insts], [x.edges for x in insts], [x.J for x in insts],
                             [x.h for x in insts], 4, [x.colour for x in insts])
    singles = [G.gtqa_create(x.n, x.edges, x.J, x.h, 4, x.colour) for x in insts]
    try:
        for k in range(1, 7):
            G.gtqa_trotter_layer(sb, k / 20, 0.1)
            G.gtqa_bp_sweep(sb, 1e-12, 100)
            for s in singles:
                G.gtqa_trotter_layer(s, k / 20, 0.1)
                G.gtqa_bp_sweep(s, 1e-12, 100)
        rb, _ = G.gtqa_marginals(sb)
        rs = np.concatenate([G.gtqa_marginals(s)[0] for s in singles])
        assert np.array_equal(rb, rs)
    finally:
        G.gtqa_destroy(sb)
        for s in singles:
            G.gtqa_destroy(s)


def _oracle_state(seed=0, layers=6, chi=4):
    inst = make_instance(16, seed)
    st = O.plus_state(inst.n, inst.edges)
    for k in range(1, layers + 1):
        tZ, tX = O.schedule(k, 20, 0.1)
        st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, chi, 1e-12, 100)
    return inst, st


def test_single_steps_from_identical_state():
    """set_state then each step alone: gates, BP (no regauge), regauge."""
    G = U.lib()
    inst, st = _oracle_state()
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour)
    try:
        n, m, C, _ = G.gtqa_sizes(s)
        Gp, Lp = O.to_padded(st, C)
        G.gtqa_set_state(s, Gp, Lp, np.zeros((2 * m, C, C), dtype=np.complex128))
        # (1) Trotter layer
        G.gtqa_trotter_layer(s, 7 / 20, 0.1)
        tZ, tX = O.schedule(7, 20, 0.1)
        O.trotter_layer(st, inst.colour, inst.J, inst.h, tZ, tX, 4)
        Gg, Lg, _ = G.gtqa_get_state(s)
        Go, Lo = O.to_padded(st, C)
        assert np.abs(Lg - Lo).max() < TOL
        assert np.abs(U.weighted_abs_gamma(Gg, Lg, st.inc) - U.weighted_abs_gamma(Go, Lo, st.inc)).max() < 1e-8
        # (2) BP from the warm start, no regauge
        it, dist, conv = G.gtqa_bp_sweep(s, 1e-12, 100, G.GTQA_BP_WARM_START)
        T = O.symmetric_gauge(st)
        msgs, it_o, hist = O.bp(st, T, O.reconstructed_messages(st), 1e-12, 100)
        _, _, Mg = G.gtqa_get_state(s)
        Mo = O.messages_to_padded(st, msgs, C)
        assert abs(it - it_o) <= 1
        assert np.abs(np.abs(Mg) - np.abs(Mo)).max() < TOL
        assert abs(dist - hist[-1]) < 1e-10
        # (3) regauge from those messages
        G.gtqa_regauge(s)
        new = O.vidal_gauge(st, T, msgs)
        rho_g, _ = G.gtqa_marginals(s)
        assert np.abs(rho_g - O.reduced_density_matrices(new)).max() < TOL
        _, Lg, _ = G.gtqa_get_state(s)
        _, Lo = O.to_padded(new, C)
        assert np.abs(Lg - Lo).max() < TOL
    finally:
        G.gtqa_destroy(s)


def test_not_converged_is_reported_and_state_stays_valid():
    G = U.lib()
    inst = make_instance(16, 1)
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour)
    try:
        G.gtqa_trotter_layer(s, 0.5, 0.1)
        it, dist, conv = G.gtqa_bp_sweep(s, 0.0, 1)
        assert it == 1 and not conv
        with pytest.raises(G.GTQAError):
            G.gtqa_bp_sweep(s, 0.0, 1, raise_not_converged=True)
        rho, sign = G.gtqa_marginals(s)
        assert np.allclose(np.trace(rho, axis1=1, axis2=2), 1.0)
        st = G.gtqa_stats(s)
        assert st["layers"] == 1 and st["gates"] == 24 and st["not_converged"] == 1
    finally:
        G.gtqa_destroy(s)


def test_stats_match_oracle_discarded_weight():
    inst = make_instance(16, 2)
    G = U.lib()
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 2, inst.colour)
    st = O.plus_state(inst.n, inst.edges)
    disc = 0.0
    logf = 0.0
    try:
        for k in range(1, 6):
            G.gtqa_trotter_layer(s, k / 10, 0.3)
            G.gtqa_bp_sweep(s, 1e-12, 100)
            tZ, tX = O.schedule(k, 10, 0.3)
            st, info = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, 2, 1e-12, 100)
            disc += info["discarded"]
            logf += info["log_fidelity"]
        sg = G.gtqa_stats(s)
        assert disc > 1e-6
        assert abs(sg["discarded_weight"] - disc) < 1e-10 * max(1.0, disc)
        assert abs(sg["log_fidelity"] - logf) < 1e-9
    finally:
        G.gtqa_destroy(s)


@pytest.mark.slow
def test_n1000_prefix_against_oracle():
    # the full-size single-instance workload (n = 1000, chi = 4, dt = 0.2, K = 3200), first layers
    inst = make_instance(1000, 0)
    out = U.run_pair(inst, 4, 3200, 0.2, 1e-8, 100, 3, check_every=3)
    assert max(out["rho"]) < 1e-9
    assert max(out["lam"]) < 1e-9


def test_many_flooding_sweeps_stay_on_the_oracle_trajectory():
    """80 sweeps with tol = 0: errors in the common phase of the messages must not grow.
    Dividing by the complex trace (App. B, unit-trace condition) keeps the flooding
    iteration identical to the oracle's; a real-part-only division lets that mode
    double every sweep on a degree-3 graph."""
    G = U.lib()
    inst, st = _oracle_state(seed=5, layers=8)
    tZ, tX = O.schedule(9, 20, 0.1)
    O.trotter_layer(st, inst.colour, inst.J, inst.h, tZ, tX, 4)
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour)
    try:
        n, m, C, _ = G.gtqa_sizes(s)
        Gp, Lp = O.to_padded(st, C)
        G.gtqa_set_state(s, Gp, Lp, np.zeros((2 * m, C, C), dtype=np.complex128))
        it, dist, conv = G.gtqa_bp_sweep(s, 0.0, 80, G.GTQA_BP_WARM_START)
        assert it == 80
        T = O.symmetric_gauge(st)
        msgs, it_o, hist = O.bp(st, T, O.reconstructed_messages(st), 0.0, 80)
        _, _, Mg = G.gtqa_get_state(s)
        Mo = O.messages_to_padded(st, msgs, C)
        assert np.abs(Mg - Mo).max() < 1e-10
        assert abs(np.trace(Mg, axis1=1, axis2=2) - 1.0).max() < 1e-13
    finally:
        G.gtqa_destroy(s)


@pytest.mark.gpu
@pytest.mark.parametrize("precision, rel, atol", [(0, 1e-6, 1e-10), (1, 2e-2, 2e-6)])
def test_residual_matches_oracle(precision, rel, atol):
    """Vidal-gauge residual R (App. C) on the device against the oracle's: after gates the
    state leaves the Vidal gauge (R up to ~4e-3 here), and the regauge brings it back down to
    the level left by the approximate BP environment.  The mixed mode is compared with an
    absolute floor for its complex64 tensors."""
    G = U.lib()
    inst = make_instance(16, 3)
    K, dt, chi = 20, 0.3, 4   # R reaches ~4e-3 by layer 8
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour, G.gtqa_options_init(precision=precision))
    try:
        st = O.plus_state(inst.n, inst.edges)
        seen, seen_after = [], []
        for k in range(1, 9):
            G.gtqa_trotter_layer(s, k / K, dt)
            tZ, tX = O.schedule(k, K, dt)
            O.trotter_layer(st, inst.colour, inst.J, inst.h, tZ, tX, chi)
            r_gpu, r_ora = G.gtqa_residual(s), O.local_orthogonality_residual(st)
            seen.append(r_ora)
            assert abs(r_gpu - r_ora) < atol + rel * r_ora, (k, r_gpu, r_ora)
            G.gtqa_bp_sweep(s, 1e-12, 100)
            T = O.symmetric_gauge(st)
            msgs, _, _ = O.bp(st, T, O.reconstructed_messages(st), 1e-12, 100)
            st = O.vidal_gauge(st, T, msgs)
            # after the regauge R is small but not zero on a loopy graph (the BP environment
            # is approximate); the complex64 storage of the mixed mode adds ~4e-7
            r_gpu, r_ora = G.gtqa_residual(s), O.local_orthogonality_residual(st)
            assert abs(r_gpu - r_ora) < atol + rel * r_ora, (k, "regauged", r_gpu, r_ora)
            seen_after.append(r_ora)
        # the first layers from the product state stay in the Vidal gauge; later ones leave it
        assert max(seen) > 1e-3, seen
        assert max(seen_after) < 1e-4 and all(x < y for x, y in zip(seen_after[2:], seen[2:])), (seen_after, seen)
    finally:
        G.gtqa_destroy(s)


@pytest.mark.gpu
@pytest.mark.parametrize("precision, tol", [(0, 1e-10), (1, 1e-5)])
def test_entropy_of_spectral_cut_matches_oracle(precision, tol):
    """Mean-field entanglement entropy (Sec. III C) of the spectral bipartition on the device
    against the oracle's, after each of 6 layers."""
    G = U.lib()
    inst = make_instance(16, 2)
    side, cut, ratio = G.gtqa_spectral_bipartition(inst.n, inst.edges)
    _, cut_o, ratio_o = O.spectral_bipartition(inst.n, inst.edges)
    assert abs(ratio - ratio_o) < 1e-12
    K, dt, chi = 20, 0.3, 4
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour, G.gtqa_options_init(precision=precision))
    try:
        st = O.plus_state(inst.n, inst.edges)
        assert G.gtqa_entropy(s, cut) == 0.0
        seen = []
        for k in range(1, 7):
            G.gtqa_trotter_layer(s, k / K, dt)
            G.gtqa_bp_sweep(s, 1e-12, 100)
            tZ, tX = O.schedule(k, K, dt)
            st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, chi, 1e-12, 100)
            s_g, s_o = G.gtqa_entropy(s, cut), O.approx_entanglement_entropy(st, cut)
            seen.append(s_o)
            assert abs(s_g - s_o) < tol * max(1.0, s_o), (k, s_g, s_o)
        assert max(seen) > 0.05   # the state is entangled across the cut by then
    finally:
        G.gtqa_destroy(s)


@pytest.mark.gpu
def test_sampling_matches_oracle():
    """BP-guided measurement sampling (Sec. IV A) on the degenerate MaxCut instance
    (J = -1, h = 0): the same order and random numbers give the oracle's bitstring,
    conditional probabilities and post-measurement marginals."""
    G = U.lib()
    inst = make_instance(12, 4, J="maxcut", h_std=0.0)
    K, dt, chi, tol, mi = 10, 0.2, 4, 1e-12, 100
    rng = np.random.default_rng(9)
    order = rng.permutation(inst.n)
    u = rng.random(inst.n)
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour)
    try:
        st = O.plus_state(inst.n, inst.edges)
        for k in range(1, K + 1):
            G.gtqa_trotter_layer(s, k / K, dt)
            G.gtqa_bp_sweep(s, tol, mi)
            tZ, tX = O.schedule(k, K, dt)
            st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, chi, tol, mi)
        x_g, p_g = G.gtqa_sample(s, order, u, tol, mi)
        x_o, p_o, st = O.sample_bitstring(st, order.tolist(), u, tol, mi)
        assert np.array_equal(x_g, x_o)
        assert np.abs(p_g - p_o).max() < 1e-8, np.abs(p_g - p_o).max()
        rho_g, _ = G.gtqa_marginals(s)
        assert np.abs(rho_g - O.reduced_density_matrices(st)).max() < 1e-8
    finally:
        G.gtqa_destroy(s)


@pytest.mark.gpu
def test_mixed_sampling_gives_a_consistent_bitstring():
    G = U.lib()
    inst = make_instance(16, 5, J="maxcut", h_std=0.0)
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour, G.gtqa_options_init(precision=G.GTQA_MIXED))
    try:
        G.gtqa_anneal(s, 1, 10, 10, 0.2, 1e-8, 100)
        rng = np.random.default_rng(3)
        order = rng.permutation(inst.n)
        x, p = G.gtqa_sample(s, order, rng.random(inst.n), 1e-8, 100)
        assert set(np.unique(x).tolist()) <= {-1, 1} and np.all(x != 0)
        assert np.all((p > 0) & (p <= 1 + 1e-6))
        rho, sign = G.gtqa_marginals(s)   # the post-measurement state is the sampled product state
        assert np.array_equal(sign, x) and np.abs(np.abs(rho[:, 0, 0].real - 0.5) - 0.5).max() < 1e-4
    finally:
        G.gtqa_destroy(s)
