"""GPU parity of the regauge policy (regauge only when the residual R exceeds a threshold,
Sec. II C): the layers regauged and the resulting marginals against the oracle's
run_with_regauge_policy (FP64, 1e-10), and the mixed mode at the two extreme thresholds."""
from __future__ import annotations

import numpy as np
import pytest

import gpu_util as U
from instances import make_instance
from oracle import gtqa_oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _oracle_thresholds(inst, args, layers):
    _, infos = O.run_with_regauge_policy(*args, -1.0, layers=layers)
    Rs = sorted(i["R"] for i in infos)
    return [-1.0, np.inf, 0.5 * (Rs[len(Rs) // 2 - 1] + Rs[len(Rs) // 2])]


@pytest.mark.parametrize("seed", [0, 1])
def test_policy_matches_oracle_fp64(seed):
    G = U.lib()
    inst = make_instance(16, seed)
    K, dt, chi, tol, mi, layers = 20, 0.1, 4, 1e-12, 200, 8
    args = (inst.n, inst.edges, inst.J, inst.h, inst.colour, K, dt, chi, tol, mi)
    for thr in _oracle_thresholds(inst, args, layers):
        st, infos = O.run_with_regauge_policy(*args, thr, layers=layers)
        s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, chi, inst.colour, G.gtqa_options_init(precision=0))
        try:
            G.gtqa_anneal_policy(s, 1, layers, K, dt, tol, mi, thr)
            reg, skip = G.gtqa_regauge_counts(s)
            n_reg = sum(i["regauged"] for i in infos)
            assert (reg, skip) == (n_reg, layers - n_reg), (thr, reg, skip, n_reg)
            rho_g, _ = G.gtqa_marginals(s)
            _, Lg, _ = G.gtqa_get_state(s)
            _, Lo = O.to_padded(st, Lg.shape[1])
            assert np.abs(rho_g - O.reduced_density_matrices(st)).max() < TOL, thr
            assert np.abs(Lg - Lo).max() < TOL, thr
        finally:
            G.gtqa_destroy(s)


def test_policy_extremes_mixed_and_batch():
    """Mixed mode at n = 1000: a negative threshold equals gtqa_anneal bit for bit; an infinite
    one skips every BP and regauge, and its marginals stay within 1e-4 of the FP64 path with the
    same policy.  A batched state applies one decision to all instances."""
    from instances import make_batch
    G = U.lib()
    inst = make_instance(1000, 0)
    K, dt, tol, mi = 3200, 0.2, 1e-8, 100
    out = {}
    for name, prec, thr in (("anneal", 1, None), ("always", 1, -1.0), ("never_mixed", 1, np.inf),
                            ("never_fp64", 0, np.inf)):
        s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour, G.gtqa_options_init(precision=prec))
        try:
            if thr is None:
                G.gtqa_anneal(s, 1, 10, K, dt, tol, mi)
            else:
                G.gtqa_anneal_policy(s, 1, 10, K, dt, tol, mi, thr)
            out[name] = (G.gtqa_get_state(s), G.gtqa_regauge_counts(s), G.gtqa_marginals(s)[0])
        finally:
            G.gtqa_destroy(s)
    for a, b in zip(out["anneal"][0], out["always"][0]):
        assert np.array_equal(a, b)
    assert out["always"][1] == (10, 0) and out["never_mixed"][1] == (0, 10)
    assert np.abs(out["never_mixed"][2] - out["never_fp64"][2]).max() < 1e-4
    insts = make_batch(4, seed=2, n_lo=50, n_hi=100)
    sb = G.gtqa_create_batch([x.n for x in insts], [x.edges for x in insts], [x.J for x in insts],
                             [x.h for x in insts], 4, [x.colour for x in insts], G.gtqa_options_init(precision=1))
    try:
        G.gtqa_anneal_policy(sb, 1, 6, 100, 0.2, 1e-8, 100, 1e-6)
        reg, skip = G.gtqa_regauge_counts(sb)
        assert reg + skip == 6
    finally:
        G.gtqa_destroy(sb)
