"""The complex64 mode (every step in FP32, including the SVDs, gauge roots and message
normalisation): against the oracle on small graphs at an FP32-sized bar, and its per-vertex
marginal error against the FP64 path at n = 1000 next to that of the mixed mode (the precision
sweep of the chi-sweep configuration)."""
from __future__ import annotations

import numpy as np
import pytest

import gpu_util as U
from instances import make_instance
from oracle import gtqa_oracle as O

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("chi", [2, 4, 8])
def test_c64_layers_follow_the_oracle(chi):
    """n = 16, 3-regular, K = 20, dt = 0.1, tol 1e-6 (above the FP32 distance floor), 8 layers:
    marginals within 1e-4 of the oracle, lambda within 1e-4."""
    G = U.lib()
    inst = make_instance(16, 3)
    K, dt, tol, mi = 20, 0.1, 1e-6, 100
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour, G.gtqa_options_init(precision=G.GTQA_C64))
    st = O.plus_state(inst.n, inst.edges)
    try:
        for k in range(1, 9):
            G.gtqa_trotter_layer(s, k / K, dt)
            G.gtqa_bp_sweep(s, tol, mi)
            tZ, tX = O.schedule(k, K, dt)
            st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, chi, 1e-12, 200)
        rho_g, _ = G.gtqa_marginals(s)
        _, Lg, _ = G.gtqa_get_state(s)
        _, Lo = O.to_padded(st, Lg.shape[1])
        assert np.abs(rho_g - O.reduced_density_matrices(st)).max() < 1e-4
        assert np.abs(Lg - Lo).max() < 1e-4
    finally:
        G.gtqa_destroy(s)


@pytest.mark.parametrize("chi", [2, 4, 8])
def test_c64_against_fp64_next_to_mixed(chi):
    """n = 1000, Gaussian J and h ~ N(0, 0.1), 12 layers of a 1000-layer schedule (dt = 0.2),
    tol 1e-8: the complex64 mode's per-vertex marginal error against the FP64 path stays below
    5e-5 (it reached 1.4e-3 at chi = 8 when FP32-noise singular values were kept), and the mixed
    mode is at least as accurate (the reason for its FP64 stages)."""
    G = U.lib()
    inst = make_instance(1000, 1, J="gauss", h_std=0.1)
    K, dt, tol, mi, layers = 1000, 0.2, 1e-8, 100, 12
    rho = {}
    for prec in (G.GTQA_FP64, G.GTQA_MIXED, G.GTQA_C64):
        s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour, G.gtqa_options_init(precision=prec))
        try:
            G.gtqa_anneal(s, 1, layers, K, dt, tol, mi)
            rho[prec], _ = G.gtqa_marginals(s)
        finally:
            G.gtqa_destroy(s)
    e_c64 = float(np.abs(rho[G.GTQA_C64] - rho[G.GTQA_FP64]).max())
    e_mix = float(np.abs(rho[G.GTQA_MIXED] - rho[G.GTQA_FP64]).max())
    print(f"chi={chi}: max |rho - rho_fp64| complex64 {e_c64:.3e}, mixed {e_mix:.3e}")
    assert e_c64 < 5e-5, e_c64
    assert e_mix <= e_c64 + 1e-12, (e_mix, e_c64)


def test_unsupported_plain_shapes_rejected():
    """Degree 4 runs on the plain kernels up to chi = 4 in every precision."""
    G = U.lib()
    inst = make_instance(10, 0, d=4)
    lib = G.load()
    import ctypes
    e = np.ascontiguousarray(inst.edges, dtype=np.int32)
    J = np.ascontiguousarray(inst.J)
    hh = np.ascontiguousarray(inst.h)
    for prec in (G.GTQA_FP64, G.GTQA_MIXED, G.GTQA_C64):
        opt = G.gtqa_options_init(precision=prec)
        h = ctypes.c_void_p()
        assert lib.gtqa_create(inst.n, inst.m, e.ctypes.data, None, J.ctypes.data, hh.ctypes.data, 8,
                               ctypes.byref(opt), ctypes.byref(h)) == G.GTQA_ERR_UNSUPPORTED


def test_c64_chi16_follows_the_oracle():
    """The complex64 mode at chi = 16 (FP32 QR, 32 x 32 Jacobi SVD and BP): n = 12, 3-regular,
    K = 20, dt = 0.3, 6 layers (bonds reach 16), within 1e-4 of the oracle on marginals and
    lambda."""
    G = U.lib()
    inst = make_instance(12, 6)
    K, dt, tol, mi = 20, 0.3, 1e-6, 100
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 16, inst.colour, G.gtqa_options_init(precision=G.GTQA_C64))
    st = O.plus_state(inst.n, inst.edges)
    try:
        n, m, C, _ = G.gtqa_sizes(s)
        assert C == 16
        for k in range(1, 7):
            G.gtqa_trotter_layer(s, k / K, dt)
            G.gtqa_bp_sweep(s, tol, mi)
            tZ, tX = O.schedule(k, K, dt)
            st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, 16, 1e-12, 200)
        rho_g, _ = G.gtqa_marginals(s)
        _, Lg, _ = G.gtqa_get_state(s)
        _, Lo = O.to_padded(st, 16)
        e_rho = float(np.abs(rho_g - O.reduced_density_matrices(st)).max())
        e_lam = float(np.abs(Lg - Lo).max())
        print(f"complex64 chi=16: marginals {e_rho:.2e}, lambda {e_lam:.2e}")
        assert e_rho < 1e-4 and e_lam < 1e-4, (e_rho, e_lam)
    finally:
        G.gtqa_destroy(s)


def test_c64_on_a_four_regular_graph_follows_the_oracle():
    """The complex64 mode on the degree-4 plain kernels (n = 10, chi = 4): within 1e-4 of the
    oracle after 6 layers."""
    G = U.lib()
    inst = make_instance(10, 2, d=4)
    K, dt, tol, mi = 20, 0.1, 1e-6, 100
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour, G.gtqa_options_init(precision=G.GTQA_C64))
    st = O.plus_state(inst.n, inst.edges)
    try:
        assert G.gtqa_max_degree(s) == 4
        for k in range(1, 7):
            G.gtqa_trotter_layer(s, k / K, dt)
            G.gtqa_bp_sweep(s, tol, mi)
            tZ, tX = O.schedule(k, K, dt)
            st, _ = O.gtqa_layer(st, inst.colour, inst.J, inst.h, tZ, tX, 4, 1e-12, 200)
        rho_g, _ = G.gtqa_marginals(s)
        assert np.abs(rho_g - O.reduced_density_matrices(st)).max() < 1e-4
    finally:
        G.gtqa_destroy(s)
