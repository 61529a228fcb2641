"""GPU parity at bond dimension 16 (the largest chi of the chi sweep): the plain FP64 kernels
against the oracle, layer by layer (bar 1e-10 on marginals and lambda)."""
from __future__ import annotations

import numpy as np
import pytest

import gpu_util as U
from instances import make_instance, make_tree_instance
from oracle import gtqa_oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.mark.parametrize("chi,kind", [(16, "regular"), (12, "regular"), (16, "tree")])
def test_chi16_layers_match_oracle(chi, kind):
    """n = 12 (3-regular) or a 14-vertex tree, J ~ N(0,1), h ~ N(0, 0.1), K = 20, dt = 0.3:
    layers of gates (truncation to chi, storage 16), BP from the warm start (tol 1e-12) and the
    regauge."""
    G = U.lib()
    inst = make_instance(12, 6) if kind == "regular" else make_tree_instance(14, 4)
    K, dt, tol, mi, layers = 20, 0.3, 1e-12, 300, 6
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour, G.gtqa_options_init(precision=G.GTQA_FP64))
    st = O.plus_state(inst.n, inst.edges)
    try:
        n, m, C, _ = G.gtqa_sizes(s)
        assert C == 16 and G.gtqa_max_degree(s) == 3
        grew = 0
        for k in range(1, layers + 1):
            G.gtqa_trotter_layer(s, k / K, dt)
            it_g, _, _ = G.gtqa_bp_sweep(s, tol, mi)
            tZ, tX = O.schedule(k, K, dt)
            st, info = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, chi, tol, mi)
            assert abs(it_g - info["bp_iters"]) <= 1, (it_g, info["bp_iters"])
            rho_g, _ = G.gtqa_marginals(s)
            _, Lg, _ = G.gtqa_get_state(s)
            _, Lo = O.to_padded(st, 16)
            assert np.abs(rho_g - O.reduced_density_matrices(st)).max() < TOL, k
            assert np.abs(Lg - Lo).max() < TOL, k
            grew = max(grew, max(l.size for l in st.lam))
        assert grew > 8   # the run reaches bond dimensions the persistent kernels do not hold
    finally:
        G.gtqa_destroy(s)


def test_chi16_anneal_symmetric_formula_and_unsupported_calls():
    G = U.lib()
    inst = make_instance(10, 2)
    K, dt, tol, mi = 20, 0.3, 1e-12, 300
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 16, inst.colour, G.gtqa_options_init(precision=G.GTQA_FP64))
    st = O.plus_state(inst.n, inst.edges)
    try:
        G.gtqa_anneal_ex(s, 1, 4, K, dt, tol, mi, G.GTQA_TROTTER_SYMMETRIC)
        for k in range(1, 5):
            t_pre, tZ, tX = O.product_formula(k, K, dt, 2)
            st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, 16, tol, mi, t_X_pre=t_pre)
        rho_g, _ = G.gtqa_marginals(s)
        assert np.abs(rho_g - O.reduced_density_matrices(st)).max() < TOL
        lib = G.load()
        Uq = np.eye(4, dtype=np.complex128).reshape(1, 4, 4).copy()
        e = np.zeros(1, dtype=np.int32)
        assert lib.gtqa_apply_gates(s, 1, e.ctypes.data, Uq.ctypes.data) == G.GTQA_ERR_UNSUPPORTED
        assert lib.gtqa_anneal_graph(s, 5, 6, K, dt, tol, mi) == G.GTQA_ERR_UNSUPPORTED
        # the state stays usable after refused calls
        G.gtqa_anneal(s, 5, 5, K, dt, tol, mi)
        assert np.isfinite(G.gtqa_marginals(s)[0]).all()
    finally:
        G.gtqa_destroy(s)


def test_chi16_single_qubit_gates_and_entropy():
    """One-qubit gates on a chi = 16 state equal the oracle's (then BP and the regauge), and the
    entropy of a cut (lambda only) matches the oracle's."""
    from instances import random_gate_inputs
    G = U.lib()
    inst = make_instance(12, 1)
    K, dt, tol, mi = 20, 0.3, 1e-12, 300
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 16, inst.colour, G.gtqa_options_init(precision=G.GTQA_FP64))
    st = O.plus_state(inst.n, inst.edges)
    try:
        G.gtqa_anneal(s, 1, 4, K, dt, tol, mi)
        for k in range(1, 5):
            tZ, tX = O.schedule(k, K, dt)
            st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, 16, tol, mi)
        _, _, v, W = random_gate_inputs(inst.n, inst.m, 0, 2 * inst.n, seed=31)
        G.gtqa_apply_single_qubit_gates(s, v, W)
        G.gtqa_bp_sweep(s, tol, mi)
        O.apply_single_qubit_gates(st, list(zip(v.tolist(), W)))
        st, _ = O.regauge(st, tol, mi)
        rho_g, _ = G.gtqa_marginals(s)
        assert np.abs(rho_g - O.reduced_density_matrices(st)).max() < TOL
        cut = np.zeros(inst.m, dtype=np.uint8)
        cut[: inst.m // 3] = 1
        assert abs(G.gtqa_entropy(s, cut) - O.approx_entanglement_entropy(st, cut.astype(bool))) < 1e-9
    finally:
        G.gtqa_destroy(s)


def test_chi16_n1000_properties_and_sampled_oracle_checks():
    """chi = 16 at n = 1000 (Gaussian J, h ~ N(0, 0.1), 4 layers of a 1000-layer schedule,
    dt = 0.2, FP64): marginals are unit-trace Hermitian PSD, and after the gates of layer 5 and
    a warm-start BP to 1e-12 the messages of sampled vertices satisfy Eq. (local_consistency) as
    evaluated by the oracle from the device's tensors and incoming messages."""
    G = U.lib()
    inst = make_instance(1000, 1)
    K, dt, tol, mi = 1000, 0.2, 1e-12, 200
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 16, inst.colour, G.gtqa_options_init(precision=G.GTQA_FP64))
    try:
        G.gtqa_anneal(s, 1, 4, K, dt, tol, mi)
        rho, _ = G.gtqa_marginals(s)
        tr = rho[:, 0, 0].real + rho[:, 1, 1].real
        assert np.abs(tr - 1).max() < 1e-12
        assert np.abs(rho - np.conj(np.swapaxes(rho, 1, 2))).max() < 1e-12
        assert np.linalg.eigvalsh(rho).min() > -1e-12
        G.gtqa_trotter_layer(s, 5 / K, dt)
        it, dist, conv = G.gtqa_bp_sweep(s, tol, mi, G.GTQA_BP_WARM_START)
        assert conv, (it, dist)
        Gg, Lg, Mg = G.gtqa_get_state(s)
    finally:
        G.gtqa_destroy(s)
    assert Lg.shape[1] == 16   # the bond storage of the chi = 16 kernels
    inc = O.incidence(inst.n, inst.edges)
    rng = np.random.default_rng(12)
    for a in rng.choice(inst.n, size=12, replace=False):
        st, msgs = U.star_state(Gg, Lg, Mg, inst.edges, inc, int(a))
        T = O.symmetric_gauge(st)
        for q in range(len(inc[a])):
            upd = O.message_update(st, T, msgs, 0, q)
            upd = upd / np.trace(upd)
            assert np.abs(upd - msgs[(q, 0)]).max() < 1e-8, (int(a), q, np.abs(upd - msgs[(q, 0)]).max())
