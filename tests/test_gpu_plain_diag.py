"""Diagnostics and measurement sampling on plain-path states (degree 4, chi = 16 and the
complex64 mode): the residual R of App. C against the oracle's, the regauge policy of Sec. II C
with the oracle's decisions and marginals, and the BP-guided sampling of Sec. IV A with the
oracle's bitstring and probabilities."""
from __future__ import annotations

import numpy as np
import pytest

import gpu_util as U
from instances import make_instance
from oracle import gtqa_oracle as O

pytestmark = pytest.mark.gpu

# name -> (instance, chi, precision, svd cut-off (0: the precision's default), R tolerance
# against the oracle's own trajectory (rel, atol after the gates, atol after the regauge), GPU
# BP tol).  R counts every kept bond index with weight one, so rounding in the tensors of bond
# indices with small lambda is amplified: at chi = 16, where bonds have spare room, both sides
# drop values below 1e-10 (with the default 1e-14 the oracle's dense SVD keeps rounding-level
# values whose singular vectors are noise); the complex64 mode's R has an FP32 floor near 1e-4
# (singular vectors of values near its 1e-7 s_0 cut-off); after the regauge R sits at the level
# of the BP convergence.  The residual kernel itself is checked against the oracle's R of the
# device's own state at 1e-12.
CASES = {
    "deg4": (lambda: make_instance(10, 4, d=4), 4, 0, 0.0, (1e-6, 1e-10, 1e-10), 1e-12),
    "chi16": (lambda: make_instance(12, 6), 16, 0, 1e-10, (1e-6, 1e-7, 1e-6), 1e-12),
    "c64": (lambda: make_instance(16, 3), 4, 2, 0.0, (1e-1, 5e-4, 5e-4), 1e-6),
}


@pytest.mark.parametrize("case", list(CASES))
def test_plain_residual_matches_oracle(case):
    """R after the gates of each layer (K = 20, dt = 0.3, 8 layers, 6 at chi = 16) and again
    after BP and the regauge: equal to the oracle's R evaluated on the device's own state (1e-12),
    and close to the oracle's R on its own trajectory."""
    make, chi, prec, cut, (rel, atol_g, atol_r), gtol = CASES[case]
    ocut = cut if cut > 0 else O.SVD_CUTOFF
    G = U.lib()
    inst = make()
    K, dt = 20, 0.3
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour,
                      G.gtqa_options_init(precision=prec, svd_cutoff=cut))

    def check(st, what, atol):
        r_gpu = G.gtqa_residual(s)
        Gg, Lg, _ = G.gtqa_get_state(s)
        r_own = O.local_orthogonality_residual(O.from_padded(inst.n, inst.edges, Gg, Lg))
        r_ora = O.local_orthogonality_residual(st)
        assert abs(r_gpu - r_own) < 1e-14 + 1e-12 * r_own, (what, r_gpu, r_own)
        assert abs(r_gpu - r_ora) < atol + rel * r_ora, (what, r_gpu, r_ora)
        return r_ora

    try:
        st = O.plus_state(inst.n, inst.edges)
        seen = []
        for k in range(1, (7 if chi == 16 else 9)):
            G.gtqa_trotter_layer(s, k / K, dt)
            tZ, tX = O.schedule(k, K, dt)
            O.trotter_layer(st, inst.colour, inst.J, inst.h, tZ, tX, chi, ocut)
            seen.append(check(st, (k, "gates"), atol_g))
            G.gtqa_bp_sweep(s, gtol, 200)
            st, _ = O.regauge(st, 1e-12, 200, svd_cutoff=ocut)
            check(st, (k, "regauged"), atol_r)
        assert max(seen) > 1e-6, seen   # the gates leave the Vidal gauge on these loopy graphs
    finally:
        G.gtqa_destroy(s)


def _split_threshold(args, layers, svd_cutoff):
    """A threshold under which the oracle regauges some layers and skips others, with every R of
    that run at least a factor 30 away from it, so that rounding cannot flip a decision."""
    for thr in (1e-8, 1e-6, 1e-10, 1e-4):
        st, infos = O.run_with_regauge_policy(*args, thr, layers=layers, svd_cutoff=svd_cutoff)
        n_reg = sum(i["regauged"] for i in infos)
        if 0 < n_reg < layers and all(i["R"] > 30 * thr or i["R"] < thr / 30 for i in infos):
            return thr, st, infos
    pytest.fail("no threshold with a clear margin")


@pytest.mark.parametrize("case", ["deg4", "chi16"])
def test_plain_policy_matches_oracle(case):
    """gtqa_anneal_policy on an FP64 plain state: for a negative, an infinite and a splitting
    threshold, the same layers are regauged as in the oracle's run_with_regauge_policy, and the
    marginals and lambda agree to 1e-10."""
    make, chi, prec, cut, _, _ = CASES[case]
    ocut = cut if cut > 0 else O.SVD_CUTOFF
    G = U.lib()
    inst = make()
    K, dt, tol, mi = 20, 0.3, 1e-12, 200
    layers = 6 if chi == 4 else 5
    args = (inst.n, inst.edges, inst.J, inst.h, inst.colour, K, dt, chi, tol, mi)
    runs = [_split_threshold(args, layers, ocut)]
    for thr in (-1.0, np.inf):
        runs.append((thr,) + O.run_with_regauge_policy(*args, thr, layers=layers, svd_cutoff=ocut))
    for thr, st, infos in runs:
        s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour,
                          G.gtqa_options_init(precision=prec, svd_cutoff=cut))
        try:
            G.gtqa_anneal_policy(s, 1, layers, K, dt, tol, mi, thr)
            reg, skip = G.gtqa_regauge_counts(s)
            n_reg = sum(i["regauged"] for i in infos)
            assert (reg, skip) == (n_reg, layers - n_reg), (thr, reg, skip, n_reg)
            rho_g, _ = G.gtqa_marginals(s)
            _, Lg, _ = G.gtqa_get_state(s)
            _, Lo = O.to_padded(st, Lg.shape[1], degree=4 if case == "deg4" else 3)
            assert np.abs(rho_g - O.reduced_density_matrices(st)).max() < 1e-10, thr
            assert np.abs(Lg - Lo).max() < 1e-10, thr
        finally:
            G.gtqa_destroy(s)


def test_plain_policy_extremes_complex64():
    """The complex64 mode: a negative threshold gives gtqa_anneal's state bit for bit, an
    infinite one skips every BP and regauge."""
    G = U.lib()
    inst = make_instance(16, 3)
    K, dt, tol, mi = 20, 0.1, 1e-6, 100
    out = {}
    for name, thr in (("anneal", None), ("always", -1.0), ("never", np.inf)):
        s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour, G.gtqa_options_init(precision=G.GTQA_C64))
        try:
            if thr is None:
                G.gtqa_anneal(s, 1, 6, K, dt, tol, mi)
            else:
                G.gtqa_anneal_policy(s, 1, 6, K, dt, tol, mi, thr)
            out[name] = (G.gtqa_get_state(s), G.gtqa_regauge_counts(s))
        finally:
            G.gtqa_destroy(s)
    for a, b in zip(out["anneal"][0], out["always"][0]):
        assert np.array_equal(a, b)
    assert out["always"][1] == (6, 0) and out["never"][1] == (0, 6)


@pytest.mark.parametrize("case", ["deg4", "chi16"])
def test_plain_sampling_matches_oracle(case):
    """BP-guided sampling on the MaxCut couplings (J = -1, h = 0), FP64 plain state: the same
    order and random numbers give the oracle's bitstring, conditional probabilities and
    post-measurement marginals."""
    G = U.lib()
    chi = 4 if case == "deg4" else 16
    inst = make_instance(10, 4, d=4, J="maxcut", h_std=0.0) if case == "deg4" else \
        make_instance(12, 4, J="maxcut", h_std=0.0)
    K, dt, tol, mi = 10, 0.2, 1e-12, 200
    layers = 6 if chi == 4 else 4
    rng = np.random.default_rng(9)
    order = rng.permutation(inst.n)
    u = rng.random(inst.n)
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour, G.gtqa_options_init(precision=0))
    try:
        st = O.plus_state(inst.n, inst.edges)
        for k in range(1, layers + 1):
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


def test_plain_sampling_complex64_gives_a_consistent_bitstring():
    G = U.lib()
    inst = make_instance(16, 5, J="maxcut", h_std=0.0)
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour, G.gtqa_options_init(precision=G.GTQA_C64))
    try:
        G.gtqa_anneal(s, 1, 10, 10, 0.2, 1e-6, 100)
        rng = np.random.default_rng(3)
        order = rng.permutation(inst.n)
        x, p = G.gtqa_sample(s, order, rng.random(inst.n), 1e-6, 100)
        assert set(np.unique(x).tolist()) <= {-1, 1} and np.all(x != 0)
        assert np.all((p > 0) & (p <= 1 + 1e-5))
        rho, sign = G.gtqa_marginals(s)   # the post-measurement state is the sampled product state
        assert np.array_equal(sign, x) and np.abs(np.abs(rho[:, 0, 0].real - 0.5) - 0.5).max() < 1e-3
    finally:
        G.gtqa_destroy(s)
