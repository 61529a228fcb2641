"""Pins of the CPU oracle against the paper's exact statements and independent routes.

Each test names the passage of arXiv:2409.12240 that fixes the expected value.
"""
import numpy as np
import pytest

import oracle_pins as P
from instances import make_instance, make_tree_instance
from oracle import gtqa_oracle as O


def test_gates_match_matrix_exponentials():
    # App. F: U_Z factors exp(-i t (J ZZ + h/D Z + h/D Z)) and U_X factors exp(-i t X)
    assert P.gate_vs_expm() < 1e-14


def test_ising_gate_has_operator_schmidt_rank_two():
    # A diagonal two-qubit gate splits into two single-qubit terms (App. E raises d_ab to at most 2 d_ab)
    W = O.ising_gate(0.7, -0.3, 1.1, 3, 2, 0.9)
    M = W.transpose(0, 2, 1, 3).reshape(4, 4)
    s = np.linalg.svd(M, compute_uv=False)
    assert np.sum(s > 1e-12 * s[0]) == 2


def test_statevector_matches_dense_exponentials():
    assert P.statevector_vs_dense() < 1e-12


def test_schedule_reading():
    # Eq. (discretizatoion), reading R1: s(t) = 1 - t/T sampled at k dt
    assert O.schedule(20, 20, 0.1) == pytest.approx((0.1, 0.0))
    tz, tx = O.schedule(1, 20, 0.1)
    assert tz == pytest.approx(0.005) and tx == pytest.approx(0.095)


@pytest.mark.parametrize("kind,n,layers", [("tree", 10, 4), ("loopy", 6, 2), ("loopy", 8, 1)])
def test_simple_update_without_truncation_is_exact(kind, n, layers):
    # App. E: absorbing lambda's and dividing them back out is an exact rewrite
    inst = make_tree_instance(n, 1) if kind == "tree" else make_instance(n, 1)
    assert P.gates_exact_without_truncation(inst, layers=layers) < 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tree_marginals_schmidt_values_and_state_are_exact(seed):
    # Sec. II B: BP is exact on trees; Sec. II C: lambda are the Schmidt coefficients
    r = P.gtqa_tree_exact(seed)
    assert r["rho"] < 1e-10 and r["lam"] < 1e-10 and r["state"] < 1e-10


def test_loopy_gtqa_state_exact_without_truncation():
    # App. D: the regauge is a gauge transformation; App. E: exact without truncation
    assert P.gtqa_loopy_state_exact(0, n=6, layers=2) < 1e-12
    assert P.gtqa_loopy_state_exact(1, n=8, layers=1) < 1e-12


def test_product_state_closed_form():
    # J = 0: each qubit evolves alone under exp(-i t_X X) exp(-i t_Z h Z) (App. F)
    assert P.product_state_closed_form() < 1e-12


def test_z2_symmetric_instance_has_zero_magnetisation():
    # h = 0: prod X commutes with H(t) and |+>^N is symmetric (Sec. III A, App. F)
    assert P.z2_symmetry() < 1e-10


def test_bp_marginals_are_gauge_covariant():
    # Eq. (local_consistency) and Eq. (partial_dens) contract ket with ket, bra with bra
    assert P.bp_gauge_covariance() < 1e-10


def test_messages_hermitian_psd_unit_trace():
    # Sec. II B, App. B: messages are Hermitian PSD, normalised to unit trace
    assert P.bp_invariants() < 1e-12


def test_flooding_and_sequential_reach_same_fixed_point():
    # App. B: both schedules iterate the same fixed-point equation
    assert P.flooding_vs_sequential() < 1e-10


def test_warm_start_is_fixed_point_after_regauge():
    # Sec. II C: for R = 0 the reconstructed messages satisfy Eq. (local_consistency)
    assert P.warm_start_fixed_point() < 1e-10


def test_residual_closed_form():
    assert P.residual_closed_form() < 1e-14


def test_residual_zero_after_regauge():
    # App. C-D: the Vidal gauge from converged messages has R = 0
    assert P.residual_after_regauge() < 1e-9


def test_regauge_changes_only_the_gauge():
    assert P.regauge_is_exact_gauge_transform() < 1e-12


def test_truncation_error_is_frobenius_norm_of_dropped_lambda():
    # Sec. II C: eps_ab = sqrt(sum_{j >= chi} lambda^2) on trees in the Vidal gauge
    assert P.truncation_frobenius() < 1e-12


def test_two_qubit_instance_exact():
    assert P.single_edge_exact() < 1e-12


def test_rounding_rule_and_objective():
    # Eq. (rounding_rule) with reading R9, Eq. (objective_function)
    rho = np.zeros((3, 2, 2), dtype=complex)
    rho[:, 0, 0] = [0.9, 0.5, 0.1]
    assert list(O.rounding(rho)) == [1, -1, -1]
    edges = np.array([[0, 1], [1, 2]])
    assert O.objective(edges, np.array([1.0, -2.0]), np.array([0.5, 0.0, -1.0]), [1, -1, 1]) == pytest.approx(-1 + 2 + 0.5 - 1)


def test_trace_norm_and_hermitian_sqrt():
    rng = np.random.default_rng(3)
    A = rng.normal(size=(5, 5)) + 1j * rng.normal(size=(5, 5))
    H = A + A.conj().T
    assert O.trace_norm(H) == pytest.approx(np.abs(np.linalg.eigvalsh(H)).sum())
    m = A @ A.conj().T
    sq, isq = O.hermitian_sqrt(m)
    assert np.abs(sq @ sq - m).max() < 1e-12
    assert np.abs(isq @ m @ isq - np.eye(5)).max() < 1e-10


def test_padded_round_trip():
    inst, st = P.loopy_state(0, n=16, layers=3)
    G, L = O.to_padded(st, 4)
    st2 = O.from_padded(st.n, st.edges, G, L)
    for a in range(st.n):
        assert np.array_equal(st.Gamma[a], st2.Gamma[a])
    tree = make_tree_instance(12, 0)
    s3 = O.plus_state(tree.n, tree.edges)
    G, L = O.to_padded(s3, 4)
    assert G.shape == (12, 2, 4, 4, 4)
    s4 = O.from_padded(tree.n, tree.edges, G, L)
    assert all(np.array_equal(a, b) for a, b in zip(s3.Gamma, s4.Gamma))


@pytest.mark.slow
def test_trace_distance_error_in_paper_band():
    # Eq. (error), Fig. 4(b): 1e-3 .. a few 1e-2 for N = 14, T = 20, chi = 4 (sanity band)
    e = P.trace_distance_band(seeds=(0, 1))
    assert 1e-4 < e < 5e-2


@pytest.mark.parametrize("seed", [0, 1])
def test_tree_one_edge_cut_entropy_is_exact(seed):
    # Sec. III C, Eq. (apprx_entropy): exact for a one-edge cut of a tree (Sec. II C)
    assert P.tree_entropy_exact(seed) < 1e-9


def test_product_state_has_zero_entropy():
    inst = make_instance(16, 0)
    st = O.plus_state(inst.n, inst.edges)
    assert O.approx_entanglement_entropy(st, np.ones(st.m, dtype=bool)) == 0.0


def test_spectral_bipartition_closed_forms_and_brute_force():
    # Eq. (bipartition): known optimal ratio cuts, and never better than the exhaustive optimum
    assert P.bipartition_closed_forms() < 1e-12
    for seed in range(3):
        assert P.bipartition_against_brute_force(seed) < 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tree_sampling_probabilities_are_born_probabilities(seed):
    # Sec. IV A sampling with Eq. (projection) and regauging; exact on trees (Sec. II B)
    assert P.tree_sampling_chain_rule(seed) < 1e-7   # BP after a projection converges to ~1e-9


def test_sampling_a_product_state_follows_its_marginals():
    # J = 0: the state stays a product, so each outcome's probability is the qubit's own marginal
    inst = make_instance(12, 0, J="ferro", h_std=0.5)
    J0 = np.zeros_like(inst.J)
    st = O.plus_state(inst.n, inst.edges)
    for k in range(1, 4):
        tZ, tX = O.schedule(k, 4, 0.5)
        st, _ = O.gtqa_layer(st, inst.colour, J0, inst.h, tZ, tX, 4, 1e-13, 100)
    rho = O.reduced_density_matrices(st)
    u = np.linspace(0.05, 0.95, inst.n)
    x, p, _ = O.sample_bitstring(st, list(range(inst.n)), u, 1e-13, 100)
    expect = np.where(u < rho[:, 0, 0].real, rho[:, 0, 0].real, rho[:, 1, 1].real)
    assert np.abs(p - expect).max() < 1e-12
    assert np.array_equal(x, np.where(u < rho[:, 0, 0].real, 1, -1))


def test_product_formula_error_orders():
    r = P.product_formula_orders(0)
    assert 3.5 < r["first"] < 4.5 and 3.5 < r["first_rev"] < 4.5, r
    assert 7.0 < r["second"] < 9.0, r
    assert 7.0 < r["randomised"] < 9.5, r


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("seed", [0, 1])
def test_tree_product_formulas_exact(order, seed):
    assert P.tree_product_formula_exact(seed, order) < 1e-10


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_general_gates_exact_on_trees(seed):
    r = P.general_gates_exact(seed)
    assert r["state"] < 1e-10 and r["rho"] < 1e-10, r


@pytest.mark.parametrize("seed", [0, 1])
def test_general_gate_truncation_keeps_optimal_schmidt_approximation(seed):
    assert P.general_gate_truncation_fidelity(seed) < 1e-10


@pytest.mark.parametrize("seed", [1, 2])
def test_gtqa_exact_on_degree_four_trees(seed):
    import numpy as np
    from instances import make_tree_instance
    assert np.bincount(make_tree_instance(10, seed, max_degree=4).edges.ravel()).max() == 4
    r = P.gtqa_tree_exact(seed, max_degree=4)
    assert r["rho"] < 1e-10 and r["lam"] < 1e-10 and r["state"] < 1e-10, r


@pytest.mark.parametrize("seed", [0, 1])
def test_regauge_policy_on_trees_stays_exact(seed):
    r = P.regauge_policy_on_trees(seed)
    assert r["never"]["regauged"] == 0 and r["never"]["rho"] < 1e-10, r
    assert r["always"]["regauged"] == 6 and r["always"]["rho"] < 1e-10, r


def test_regauge_policy_on_loopy_graphs():
    r = P.regauge_policy_on_loopy_graphs(0)
    assert r["all_regauged"] and r["rho"] == 0.0 and r["none_regauged"], r
    assert r["threshold_rule"] and r["some_skipped"], r
