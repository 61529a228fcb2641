"""GPU parity at the shapes of the other workloads: the batched uneven configuration
(256 instances, n uniform over even values in [50, 1000], chi = 4, dt = 0.05), the
bond-dimension sweep at n = 1000 (chi in {2, 4, 8}, Gaussian, ferromagnetic and MaxCut
couplings, FP64 against mixed), and the n = 100000, chi = 8 scale configuration
(properties and oracle-computed local checks on sampled vertices)."""
from __future__ import annotations

import numpy as np
import pytest

import gpu_util as U
from instances import make_batch, make_instance
from oracle import gtqa_oracle as O

pytestmark = pytest.mark.gpu


def _clear_signs_equal(rho_a, rho_b):
    clear = np.abs(rho_b[:, 0, 0].real - 0.5) > 1e-3
    sa = np.where(rho_a[:, 0, 0].real > 0.5, 1, -1)
    sb = np.where(rho_b[:, 0, 0].real > 0.5, 1, -1)
    return bool(np.array_equal(sa[clear], sb[clear]))


def test_batched_uneven_instances_match_single_runs_and_oracle():
    """256 instances in one batched state (one launch per phase per layer) against single-
    instance FP64 GPU runs of 8 sampled instances and the oracle on the two smallest."""
    G = U.lib()
    insts = make_batch(256, seed=0)
    K, dt, chi, tol, mi, layers = 400, 0.05, 4, 1e-8, 100, 8
    sb = G.gtqa_create_batch([x.n for x in insts], [x.edges for x in insts], [x.J for x in insts],
                             [x.h for x in insts], chi, [x.colour for x in insts],
                             G.gtqa_options_init(precision=G.GTQA_MIXED))
    try:
        G.gtqa_anneal(sb, 1, layers, K, dt, tol, mi)
        rho_b, _ = G.gtqa_marginals(sb)
    finally:
        G.gtqa_destroy(sb)
    off = np.concatenate([[0], np.cumsum([x.n for x in insts])])
    rng = np.random.default_rng(5)
    sample = sorted(rng.choice(len(insts), size=8, replace=False).tolist())
    for b in sample:
        x = insts[b]
        s = G.gtqa_create(x.n, x.edges, x.J, x.h, chi, x.colour, G.gtqa_options_init(precision=G.GTQA_FP64))
        try:
            G.gtqa_anneal(s, 1, layers, K, dt, tol, mi)
            rho_s, _ = G.gtqa_marginals(s)
        finally:
            G.gtqa_destroy(s)
        rb = rho_b[off[b]:off[b + 1]]
        assert np.abs(rb - rho_s).max() < 1e-4, (b, np.abs(rb - rho_s).max())
        assert _clear_signs_equal(rb, rho_s), b
    for b in np.argsort([x.n for x in insts])[:2]:
        x = insts[b]
        st = O.plus_state(x.n, x.edges)
        for k in range(1, layers + 1):
            tZ, tX = O.schedule(k, K, dt)
            st, _ = O.gtqa_layer(st, x.colour, x.J, x.h, tZ, tX, chi, tol, mi)
        rho_o = O.reduced_density_matrices(st)
        rb = rho_b[off[b]:off[b + 1]]
        assert np.abs(rb - rho_o).max() < 1e-4, (int(b), np.abs(rb - rho_o).max())


@pytest.mark.parametrize("chi", [2, 4, 8])
@pytest.mark.parametrize("J", ["ferro", "maxcut", "gauss"])
def test_chi_sweep_mixed_against_fp64(chi, J):
    """n = 1000: J = +1 or J = -1 (the MaxCut couplings of Sec. IV A) with h = 0, both
    degenerate, and Gaussian J, h; the mixed path against the FP64 path, per vertex, after 12
    layers of a 1000-layer schedule (dt = 0.2)."""
    G = U.lib()
    inst = make_instance(1000, 1, J=J, h_std=0.1 if J == "gauss" else 0.0)
    K, dt, tol, mi, layers = 1000, 0.2, 1e-8, 100, 12
    rho = {}
    for prec in (G.GTQA_FP64, G.GTQA_MIXED):
        s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour, G.gtqa_options_init(precision=prec))
        try:
            G.gtqa_anneal(s, 1, layers, K, dt, tol, mi)
            rho[prec], _ = G.gtqa_marginals(s)
        finally:
            G.gtqa_destroy(s)
    err = np.abs(rho[G.GTQA_MIXED] - rho[G.GTQA_FP64]).max()
    assert err < 1e-4, err
    if J == "gauss":
        assert _clear_signs_equal(rho[G.GTQA_MIXED], rho[G.GTQA_FP64])


def test_scale_n100000_chi8_properties_and_sampled_oracle_checks():
    """n = 100000, chi = 8, mixed, one layer of a 500-layer schedule (dt = 0.05): marginals
    are unit-trace Hermitian PSD, the Vidal residual after the regauge is small, and after a
    further warm-start BP the messages of sampled vertices satisfy Eq. (local_consistency)
    as evaluated by the oracle from the device's tensors and incoming messages."""
    G = U.lib()
    inst = make_instance(100000, 2)
    K, dt, chi, tol, mi = 500, 0.05, 8, 1e-8, 100
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour, G.gtqa_options_init(precision=G.GTQA_MIXED))
    try:
        G.gtqa_anneal(s, 1, 1, K, dt, tol, mi)
        rho, _ = G.gtqa_marginals(s)
        tr = rho[:, 0, 0].real + rho[:, 1, 1].real
        assert np.abs(tr - 1).max() < 1e-6
        assert np.abs(rho - np.conj(np.swapaxes(rho, 1, 2))).max() < 1e-6
        assert np.linalg.eigvalsh(rho).min() > -1e-6
        assert G.gtqa_residual(s) < 1e-4
        G.gtqa_trotter_layer(s, 2 / K, dt)
        it, dist, conv = G.gtqa_bp_sweep(s, tol, mi, G.GTQA_BP_WARM_START)
        assert conv, (it, dist)
        Gg, Lg, Mg = G.gtqa_get_state(s)
    finally:
        G.gtqa_destroy(s)
    inc = O.incidence(inst.n, inst.edges)
    rng = np.random.default_rng(11)
    for a in rng.choice(inst.n, size=16, replace=False):
        st, msgs = U.star_state(Gg, Lg, Mg, inst.edges, inc, int(a))
        T = O.symmetric_gauge(st)
        for q in range(len(inc[a])):
            upd = O.message_update(st, T, msgs, 0, q)
            upd = upd / np.trace(upd)
            assert np.abs(upd - msgs[(q, 0)]).max() < 1e-5, (int(a), q, np.abs(upd - msgs[(q, 0)]).max())
