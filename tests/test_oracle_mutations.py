"""Planted mistakes in the oracle must be caught by at least one pin.

Each test monkeypatches one plausible error into the oracle (on the CPU) and
asserts that a pin then fails.  This guards against pins that pass vacuously.
"""
import types

import numpy as np
import pytest

import oracle_pins as P
from instances import make_instance, make_tree_instance
from oracle import gtqa_oracle as O


def _np_with(**linalg_overrides):
    lin = types.SimpleNamespace(**{k: getattr(np.linalg, k) for k in dir(np.linalg) if not k.startswith("_")})
    for k, v in linalg_overrides.items():
        setattr(lin, k, v)
    proxy = types.SimpleNamespace(**{k: getattr(np, k) for k in dir(np) if not k.startswith("__")})
    proxy.linalg = lin
    return proxy


def test_transposed_right_singular_vectors_caught(monkeypatch):
    svd = np.linalg.svd

    def bad_svd(a, *args, **kw):
        r = svd(a, *args, **kw)
        if isinstance(r, tuple) or hasattr(r, "U"):
            U, s, Vh = r
            return U, s, Vh.conj()     # Gamma_b = V^T instead of V^*
        return r
    monkeypatch.setattr(O, "np", _np_with(svd=bad_svd))
    assert P.gates_exact_without_truncation(make_instance(6, 1), layers=2) > 1e-6


def test_dropped_field_term_caught(monkeypatch):
    orig = O.ising_gate
    monkeypatch.setattr(O, "ising_gate", lambda J, ha, hb, Da, Db, t: orig(J, 0.0, 0.0, Da, Db, t))
    assert P.gates_exact_without_truncation(make_tree_instance(10, 1), layers=3) > 1e-6


def test_wrong_sign_mixing_gate_caught(monkeypatch):
    orig = O.mixing_gate
    monkeypatch.setattr(O, "mixing_gate", lambda t: orig(-t))
    assert P.product_state_closed_form() > 1e-6


def test_transposed_incoming_message_caught(monkeypatch):
    orig = O.message_update

    def bad(st, T, msgs, a, e):
        return orig(st, T, {k: v.T for k, v in msgs.items()}, a, e)
    monkeypatch.setattr(O, "message_update", bad)
    assert P.bp_gauge_covariance() > 1e-6


def test_transposed_inverse_square_root_caught(monkeypatch):
    orig = O.hermitian_sqrt

    def bad(m, cutoff=O.EIG_CUTOFF):
        sq, isq = orig(m, cutoff)
        return sq, isq.T
    monkeypatch.setattr(O, "hermitian_sqrt", bad)
    assert P.regauge_is_exact_gauge_transform() > 1e-6


def test_swapped_schedule_angles_caught(monkeypatch):
    orig = O.schedule
    monkeypatch.setattr(O, "schedule", lambda k, K, dt: orig(k, K, dt)[::-1])
    assert P.gtqa_tree_exact(0)["rho"] > 1e-6


def test_printed_sqrt_warm_start_is_not_a_fixed_point(monkeypatch):
    # reading R3: the printed lambda^{1/2} form is not the fixed point of Eq. (local_consistency)
    orig = O.reconstructed_messages
    monkeypatch.setattr(O, "reconstructed_messages", lambda st, paper_sqrt_warmstart=False: orig(st, True))
    assert P.warm_start_fixed_point() > 1e-6


def test_wrong_symmetric_split_caught(monkeypatch):
    def bad(st):
        T = []
        for a in range(st.n):
            t = st.Gamma[a]
            for k, e in enumerate(st.inc[a]):
                t = O._scale_slot(t, k, st.lam[e])   # lambda instead of lambda^{1/2}
            T.append(t)
        return T
    monkeypatch.setattr(O, "symmetric_gauge", bad)
    assert P.gtqa_tree_exact(0)["rho"] > 1e-6


def test_lopsided_symmetric_formula_caught(monkeypatch):
    orig = O.product_formula

    def bad(k, K, dt, order=1, reverse=False):
        p, z, q = orig(k, K, dt, order, reverse)
        return (p, z, 2 * q) if order == 2 else (p, z, q)    # t_X/2 before, t_X after
    monkeypatch.setattr(O, "product_formula", bad)
    r = P.product_formula_orders(0)
    assert not (7.0 < r["second"] < 9.0)


def test_dropped_leading_mixing_caught(monkeypatch):
    orig = O.trotter_layer

    def bad(st, colour, J, h, t_Z, t_X, chi, svd_cutoff=O.SVD_CUTOFF, t_X_pre=0.0):
        return orig(st, colour, J, h, t_Z, t_X, chi, svd_cutoff, 0.0)
    monkeypatch.setattr(O, "trotter_layer", bad)
    assert P.tree_product_formula_exact(0, 2) > 1e-6


def test_transposed_two_qubit_gate_caught(monkeypatch):
    orig = O.simple_update

    def bad(st, e, W, chi, svd_cutoff=O.SVD_CUTOFF):
        return orig(st, e, np.transpose(W, (2, 3, 0, 1)), chi, svd_cutoff)
    monkeypatch.setattr(O, "simple_update", bad)
    assert P.general_gates_exact(0)["state"] > 1e-6


def test_swapped_gate_qubits_caught(monkeypatch):
    orig = O.simple_update

    def bad(st, e, W, chi, svd_cutoff=O.SVD_CUTOFF):
        return orig(st, e, np.transpose(W, (1, 0, 3, 2)), chi, svd_cutoff)
    monkeypatch.setattr(O, "simple_update", bad)
    assert P.general_gates_exact(0)["state"] > 1e-6


def test_truncation_keeping_the_smallest_values_caught(monkeypatch):
    svd = np.linalg.svd

    def bad_svd(a, *args, **kw):
        r = svd(a, *args, **kw)
        if isinstance(r, tuple) or hasattr(r, "U"):
            U, s, Vh = r
            k = int(np.sum(s > 1e-12 * s[0]))
            idx = np.r_[np.arange(k)[::-1], np.arange(k, s.size)]
            return U[:, idx], s[idx], Vh[idx, :]
        return r
    monkeypatch.setattr(O, "np", _np_with(svd=bad_svd))
    assert P.general_gate_truncation_fidelity(0) > 1e-6


def test_frobenius_instead_of_trace_norm_in_residual_caught(monkeypatch):
    """R of App. C uses the trace norm; a Frobenius norm leaves R = 0 after the regauge but
    changes the closed-form value."""
    monkeypatch.setattr(O, "trace_norm", lambda A: float(np.linalg.norm(A)))
    assert P.residual_closed_form() > 1e-3


def test_lambda_instead_of_lambda_squared_in_residual_caught(monkeypatch):
    """Weighting the other slots by lambda instead of lambda^2 (App. C)."""
    orig = O._scale_slot

    def bad(t, slot, vec):
        return orig(t, slot, np.sqrt(np.abs(vec)))
    monkeypatch.setattr(O, "_scale_slot", bad)
    assert P.residual_closed_form() > 1e-3

