"""Mixed-precision path (complex64 tensors and BP contractions; FP64 QR/SVD, gauge
roots and normalisation) against the FP64 oracle: <= 1e-4 absolute on marginals and
the same sign read-out wherever |rho_00 - 1/2| > 1e-3."""
import numpy as np
import pytest

import gpu_util as U
from instances import make_instance, make_tree_instance

pytestmark = pytest.mark.gpu


def _check(out, rho_tol=1e-4):
    assert max(out["rho"]) < rho_tol, out["rho"]
    assert max(out["lam"]) < 1e-3, out["lam"]
    rho_g, sign_g = out["rho_gpu"]
    from oracle import gtqa_oracle as O
    rho_o = O.reduced_density_matrices(out["state"])
    sign_o = O.rounding(rho_o)
    clear = np.abs(rho_o[:, 0, 0].real - 0.5) > 1e-3
    assert np.array_equal(sign_g[clear], sign_o[clear])


@pytest.mark.parametrize("seed", range(3))
def test_mixed_regular_n16_chi4(seed):
    inst = make_instance(16, seed)
    out = U.run_pair(inst, 4, 20, 0.1, 1e-12, 100, 20, precision=1)
    _check(out)


@pytest.mark.parametrize("chi", [2, 8])
def test_mixed_other_chi(chi):
    inst = make_instance(16, 11)
    out = U.run_pair(inst, chi, 20, 0.1, 1e-12, 100, 12, precision=1)
    _check(out)


def test_mixed_tree():
    inst = make_tree_instance(16, 2)
    out = U.run_pair(inst, 4, 20, 0.1, 1e-12, 100, 10, precision=1)
    _check(out)


def test_mixed_bp_reaches_tight_tolerance():
    """The m0 + delta form keeps the FP32 noise proportional to |delta|, so BP in the
    mixed mode converges to dist/|E| < 1e-10 like the FP64 path."""
    G = U.lib()
    inst = make_instance(16, 4)
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour, G.gtqa_options_init(precision=1))
    try:
        for k in range(1, 9):
            G.gtqa_trotter_layer(s, k / 20, 0.1)
            it, d, conv = G.gtqa_bp_sweep(s, 1e-10, 100)
            assert conv and d < 1e-10, (k, it, d)
    finally:
        G.gtqa_destroy(s)
