"""GPU parity for the product formulas of Sec. V (symmetric and randomised first order),
arbitrary one- and two-qubit gates (Sec. II D, App. E) and heavy-hexagon lattices, against
the oracle (FP64 bar 1e-10) and, for the mixed mode, against the FP64 path."""
from __future__ import annotations

import numpy as np
import pytest

import gpu_util as U
from instances import make_heavy_hex_instance, make_instance, make_tree_instance, random_gate_inputs
from oracle import gtqa_oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _create(G, inst, chi, precision):
    return G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour, G.gtqa_options_init(precision=precision))


def _lam_err(G, s, st):
    _, Lg, _ = G.gtqa_get_state(s)
    _, Lo = O.to_padded(st, Lg.shape[1])
    return float(np.abs(Lg - Lo).max())


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("seed", [0, 1])
def test_product_formulas_match_oracle(order, seed):
    """gtqa_anneal_ex layer by layer against the oracle's run with the same formula (and, for
    the first order, the same per-layer reversal draws)."""
    G = U.lib()
    inst = make_instance(16, seed)
    K, dt, chi, tol, mi, layers = 20, 0.1, 4, 1e-12, 100, 10
    rng = np.random.default_rng(100 + seed)
    rev = rng.integers(0, 2, size=layers).astype(np.uint8) if order == 1 else None
    s = _create(G, inst, chi, G.GTQA_FP64)
    st = O.plus_state(inst.n, inst.edges)
    try:
        for k in range(1, layers + 1):
            G.gtqa_anneal_ex(s, k, k, K, dt, tol, mi, order, None if rev is None else rev[k - 1:k])
            t_pre, tZ, tX = O.product_formula(k, K, dt, order, bool(rev[k - 1]) if rev is not None else False)
            st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, chi, tol, mi, t_X_pre=t_pre)
            rho_g, _ = G.gtqa_marginals(s)
            assert np.abs(rho_g - O.reduced_density_matrices(st)).max() < TOL, k
            assert _lam_err(G, s, st) < TOL, k
    finally:
        G.gtqa_destroy(s)


def test_anneal_ex_first_order_equals_anneal_and_split_equals_layer():
    G = U.lib()
    inst = make_instance(32, 3)
    K, dt, chi, tol, mi = 50, 0.2, 4, 1e-10, 100
    out = []
    for use_ex in (False, True):
        s = _create(G, inst, chi, G.GTQA_MIXED)
        try:
            if use_ex:
                G.gtqa_anneal_ex(s, 1, 6, K, dt, tol, mi, G.GTQA_TROTTER_FIRST, np.zeros(6, np.uint8))
            else:
                G.gtqa_anneal(s, 1, 6, K, dt, tol, mi)
            out.append(G.gtqa_get_state(s))
        finally:
            G.gtqa_destroy(s)
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    out = []
    for split in (False, True):
        s = _create(G, inst, chi, G.GTQA_FP64)
        try:
            for k in (1, 2, 3):
                if split:
                    G.gtqa_trotter_split(s, dt * (k / K), 0.0, dt * (1 - k / K))
                else:
                    G.gtqa_trotter_layer(s, k / K, dt)
                G.gtqa_bp_sweep(s, tol, mi)
            out.append(G.gtqa_get_state(s))
        finally:
            G.gtqa_destroy(s)
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_product_formula_arguments_rejected():
    G = U.lib()
    inst = make_instance(16, 0)
    s = _create(G, inst, 4, G.GTQA_FP64)
    try:
        lib = G.load()
        rv = np.zeros(2, np.uint8)
        assert lib.gtqa_anneal_ex(s, 1, 2, 10, 0.1, 1e-8, 10, 2, rv.ctypes.data) == G.GTQA_ERR_INVALID_ARG
        assert lib.gtqa_anneal_ex(s, 1, 2, 10, 0.1, 1e-8, 10, 3, None) == G.GTQA_ERR_INVALID_ARG
        assert lib.gtqa_anneal_ex(s, 2, 1, 10, 0.1, 1e-8, 10, 1, None) == G.GTQA_ERR_INVALID_ARG
        assert lib.gtqa_trotter_split(s, float("nan"), 0.0, 0.1) == G.GTQA_ERR_INVALID_ARG
    finally:
        G.gtqa_destroy(s)


def _gate_rounds(inst, chi, rounds, seed):
    out = []
    for r in range(rounds):
        e, Uq, v, W = random_gate_inputs(inst.n, inst.m, 2 * inst.m, inst.n, seed=1000 * seed + r)
        out.append((e, Uq, v, W))
    return out


def _run_gates_gpu(G, s, rounds, tol, mi, regauge=True):
    for e, Uq, v, W in rounds:
        G.gtqa_apply_gates(s, e, Uq)
        G.gtqa_apply_single_qubit_gates(s, v, W)
        if regauge:
            G.gtqa_bp_sweep(s, tol, mi)


def _run_gates_oracle(st, rounds, chi, tol, mi, regauge=True):
    for e, Uq, v, W in rounds:
        O.apply_gates(st, list(zip(e.tolist(), Uq)), chi)
        O.apply_single_qubit_gates(st, list(zip(v.tolist(), W)))
        if regauge:
            st, _ = O.regauge(st, tol, mi)
    return st


@pytest.mark.parametrize("chi", [2, 4, 8])
@pytest.mark.parametrize("kind", ["regular", "tree"])
def test_general_gates_match_oracle(chi, kind):
    """Haar-random gates on every edge (twice per round, in random order, repeats allowed)
    and on every vertex, with truncation to chi, then BP and the regauge; lambda, the
    marginals and the contracted state against the oracle."""
    G = U.lib()
    inst = make_instance(12, 5) if kind == "regular" else make_tree_instance(12, 5)
    tol, mi = 1e-12, 200
    rounds = _gate_rounds(inst, chi, 2, seed=chi)
    s = _create(G, inst, chi, G.GTQA_FP64)
    try:
        # the gates alone, before any regauge: lambda and the represented state
        G.gtqa_apply_gates(s, rounds[0][0], rounds[0][1])
        st = O.plus_state(inst.n, inst.edges)
        O.apply_gates(st, list(zip(rounds[0][0].tolist(), rounds[0][1])), chi)
        assert _lam_err(G, s, st) < TOL
        Gg, Lg, _ = G.gtqa_get_state(s)
        psi_g = O.to_statevector(O.from_padded(inst.n, inst.edges, Gg, Lg)).reshape(-1)
        psi_o = O.to_statevector(st).reshape(-1)
        ov = abs(np.vdot(psi_g, psi_o)) / (np.linalg.norm(psi_g) * np.linalg.norm(psi_o))
        assert abs(1 - ov) < TOL and abs(np.linalg.norm(psi_g) - np.linalg.norm(psi_o)) < TOL
        # then single-qubit gates, regauge, and a second round
        G.gtqa_apply_single_qubit_gates(s, rounds[0][2], rounds[0][3])
        G.gtqa_bp_sweep(s, tol, mi)
        O.apply_single_qubit_gates(st, list(zip(rounds[0][2].tolist(), rounds[0][3])))
        st, _ = O.regauge(st, tol, mi)
        _run_gates_gpu(G, s, rounds[1:], tol, mi)
        st = _run_gates_oracle(st, rounds[1:], chi, tol, mi)
        rho_g, _ = G.gtqa_marginals(s)
        assert np.abs(rho_g - O.reduced_density_matrices(st)).max() < TOL
        assert _lam_err(G, s, st) < TOL
        stats = G.gtqa_stats(s)
        assert stats["gates"] >= sum(r[0].size for r in rounds)
    finally:
        G.gtqa_destroy(s)


@pytest.mark.parametrize("chi", [2, 4, 8])
def test_general_gates_mixed_against_fp64(chi):
    G = U.lib()
    inst = make_instance(64, 8)
    rounds = _gate_rounds(inst, chi, 3, seed=50 + chi)
    res = {}
    for prec in (G.GTQA_FP64, G.GTQA_MIXED):
        s = _create(G, inst, chi, prec)
        try:
            _run_gates_gpu(G, s, rounds, 1e-10, 200)
            rho, _ = G.gtqa_marginals(s)
            res[prec] = (rho, G.gtqa_get_state(s)[1])
        finally:
            G.gtqa_destroy(s)
    assert np.abs(res[G.GTQA_MIXED][0] - res[G.GTQA_FP64][0]).max() < 1e-4
    assert np.abs(res[G.GTQA_MIXED][1] - res[G.GTQA_FP64][1]).max() < 1e-4


def test_single_qubit_gates_compose_in_list_order():
    """Repeated one-qubit gates on a vertex: the device result equals the oracle's
    sequential application element by element (FP64)."""
    G = U.lib()
    inst = make_instance(16, 2)
    s = _create(G, inst, 4, G.GTQA_FP64)
    try:
        G.gtqa_anneal(s, 1, 3, 20, 0.2, 1e-12, 100)
        G0, L0, M0 = G.gtqa_get_state(s)
        e, Uq, v, W = random_gate_inputs(inst.n, inst.m, 0, 3 * inst.n, seed=77)
        G.gtqa_apply_single_qubit_gates(s, v, W)
        Gg, _, _ = G.gtqa_get_state(s)
    finally:
        G.gtqa_destroy(s)
    Go = G0.copy()
    for a, w in zip(v.tolist(), W):
        Go[a] = np.tensordot(w, Go[a], axes=([1], [0]))
    # relative to each vertex tensor's scale (Gamma = U / prod lambda reaches 1e5 here)
    scale = np.abs(Go).reshape(Go.shape[0], -1).max(axis=1)
    assert (np.abs(Gg - Go).reshape(Go.shape[0], -1).max(axis=1) <= 1e-14 * scale + 1e-300).all()


def test_gate_arguments_rejected():
    G = U.lib()
    inst = make_instance(16, 0)
    s = _create(G, inst, 4, G.GTQA_FP64)
    try:
        lib = G.load()
        Uq = np.eye(4, dtype=np.complex128).reshape(1, 4, 4).copy()
        bad = np.array([inst.m], dtype=np.int32)
        assert lib.gtqa_apply_gates(s, 1, bad.ctypes.data, Uq.ctypes.data) == G.GTQA_ERR_INVALID_ARG
        Un = Uq.copy()
        Un[0, 1, 2] = np.nan
        ok = np.array([0], dtype=np.int32)
        assert lib.gtqa_apply_gates(s, 1, ok.ctypes.data, Un.ctypes.data) == G.GTQA_ERR_INVALID_ARG
        assert lib.gtqa_apply_gates(s, -1, None, None) == G.GTQA_ERR_INVALID_ARG
        W = np.eye(2, dtype=np.complex128).reshape(1, 2, 2).copy()
        badv = np.array([inst.n], dtype=np.int32)
        assert lib.gtqa_apply_single_qubit_gates(s, 1, badv.ctypes.data, W.ctypes.data) == G.GTQA_ERR_INVALID_ARG
        # rejected calls leave the state usable
        G.gtqa_apply_gates(s, ok, Uq)
        assert G.gtqa_bp_sweep(s, 1e-10, 50)[2]
    finally:
        G.gtqa_destroy(s)


@pytest.mark.parametrize("precision", [0, 1])
def test_heavy_hex_anneal_matches_oracle(precision):
    """Heavy-hexagon lattice (degree 2 and 3, shortest loop 12): FP64 parity with the oracle,
    and the mixed mode within 1e-4 of it."""
    inst = make_heavy_hex_instance(3, 9, seed=0)
    out = U.run_pair(inst, 4, 20, 0.1, 1e-12, 100, 10, precision=precision)
    tol = TOL if precision == 0 else 1e-4
    assert max(out["rho"]) < tol, out["rho"]
    assert max(out["lam"]) < tol, out["lam"]
