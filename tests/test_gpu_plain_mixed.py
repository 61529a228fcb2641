"""The mixed precision on the plain path (degree-4 graphs and chi = 16): complex64 Gamma and T,
messages held as delta = m - m0 in complex64 with FP32 contractions of the delta terms; FP64
QR/SVD in the gates, FP64 warm-start defect, normalisation and trace norms, FP64
eigen-decompositions and SVD in the regauge.  Against the oracle (1e-4 on marginals
and lambda, as for the persistent mixed path), against the FP64 plain path, the state round trip,
and the residual kernel on a mixed state against the oracle's R of that state."""
from __future__ import annotations

import numpy as np
import pytest

import gpu_util as U
from instances import make_instance
from oracle import gtqa_oracle as O

pytestmark = pytest.mark.gpu

CASES = {
    "deg4_chi4": (lambda: make_instance(10, 4, d=4), 4, 4),
    "deg4_chi2": (lambda: make_instance(10, 1, d=4), 2, 4),
    "chi16": (lambda: make_instance(12, 6), 16, 3),
}


@pytest.mark.parametrize("case", list(CASES))
def test_plain_mixed_follows_the_oracle(case):
    """K = 20, dt = 0.3 (chi = 16: 6 layers, bonds reach 16) or dt = 0.1 (degree 4: 6 layers);
    GPU BP tol 1e-8, oracle 1e-12."""
    make, chi, D = CASES[case]
    G = U.lib()
    inst = make()
    K, dt = 20, (0.3 if chi == 16 else 0.1)
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour, G.gtqa_options_init(precision=G.GTQA_MIXED))
    st = O.plus_state(inst.n, inst.edges)
    try:
        assert G.gtqa_max_degree(s) == D
        for k in range(1, 7):
            G.gtqa_trotter_layer(s, k / K, dt)
            G.gtqa_bp_sweep(s, 1e-8, 200)
            tZ, tX = O.schedule(k, K, dt)
            st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, chi, 1e-12, 200)
        rho_g, _ = G.gtqa_marginals(s)
        _, Lg, _ = G.gtqa_get_state(s)
        _, Lo = O.to_padded(st, Lg.shape[1], degree=D)
        e_rho = float(np.abs(rho_g - O.reduced_density_matrices(st)).max())
        e_lam = float(np.abs(Lg - Lo).max())
        print(f"mixed plain {case}: marginals {e_rho:.2e}, lambda {e_lam:.2e}")
        assert e_rho < 1e-4 and e_lam < 1e-4, (e_rho, e_lam)
    finally:
        G.gtqa_destroy(s)


def test_plain_mixed_state_round_trip_and_residual():
    """get_state / set_state reproduce the marginals bit for bit on a mixed plain state (the
    messages are returned as m0 + delta in complex128, with unit trace), and the residual kernel
    equals the oracle's R of the device's own state."""
    G = U.lib()
    inst = make_instance(10, 4, d=4)
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour, G.gtqa_options_init(precision=G.GTQA_MIXED))
    try:
        G.gtqa_anneal(s, 1, 4, 20, 0.3, 1e-8, 200)
        G.gtqa_trotter_layer(s, 5 / 20, 0.3)
        Gm, L, M = G.gtqa_get_state(s)
        r_gpu = G.gtqa_residual(s)
        r_own = O.local_orthogonality_residual(O.from_padded(inst.n, inst.edges, Gm, L))
        assert abs(r_gpu - r_own) < 1e-14 + 1e-12 * r_own, (r_gpu, r_own)
        G.gtqa_bp_sweep(s, 1e-8, 200)
        rho0, _ = G.gtqa_marginals(s)
        Gm, L, M = G.gtqa_get_state(s)
        G.gtqa_set_state(s, Gm, L, M)
        rho1, _ = G.gtqa_marginals(s)
        assert np.array_equal(rho0, rho1)
        assert np.abs(np.trace(M, axis1=1, axis2=2) - 1).max() < 1e-5   # unit-trace messages
    finally:
        G.gtqa_destroy(s)


@pytest.mark.parametrize("chi,d", [(16, 3), (4, 4)])
def test_plain_mixed_against_fp64_at_n1000_scale(chi, d):
    """n = 1000 (chi = 16, 3-regular) or n = 200 (4-regular, chi = 4), Gaussian J, h ~ N(0, 0.1),
    K = 1000, dt = 0.2, 8 layers, tol 1e-8: the mixed plain path within 1e-4 of the FP64 plain
    path per vertex, with the same clear signs."""
    G = U.lib()
    inst = make_instance(1000 if d == 3 else 200, 1, d=d)
    rho = {}
    for prec in (G.GTQA_FP64, G.GTQA_MIXED):
        s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour, G.gtqa_options_init(precision=prec))
        try:
            G.gtqa_anneal(s, 1, 8, 1000, 0.2, 1e-8, 100)
            rho[prec] = G.gtqa_marginals(s)
        finally:
            G.gtqa_destroy(s)
    err = float(np.abs(rho[G.GTQA_MIXED][0] - rho[G.GTQA_FP64][0]).max())
    print(f"mixed vs FP64, chi={chi}, degree {d}: {err:.2e}")
    assert err < 1e-4, err
    ref = rho[G.GTQA_FP64][0]
    clear = np.abs(ref[:, 0, 0].real - 0.5) > 1e-3
    assert np.array_equal(rho[G.GTQA_MIXED][1][clear], rho[G.GTQA_FP64][1][clear])
