"""The algebra behind the delta form that the mixed-mode BP kernels use (persistent and plain
paths), checked with the oracle's own message update of Eq. (local_consistency): the update is
linear in each incoming message, so with m = m0 + delta

    F(m_1, ..., m_k) - F(m0_1, ..., m0_k) = sum_c F(m0_1, ..., m0_{c-1}, delta_c, m_{c+1}, ..., m_k),

and the normalised new message satisfies

    m' - m0 = (D0 + F_delta - m0 tr F_delta) / (t0 + tr F_delta),  D0 = F0 - t0 m0,  t0 = tr F0.

Both are exact identities; they are checked to rounding on a degree-4 star (three incoming
messages per outgoing one, as in the degree-4 kernels) and a degree-3 star."""
import numpy as np
import pytest

from oracle import gtqa_oracle as O


def _star(k, d, seed):
    rng = np.random.default_rng(seed)
    edges = np.array([[0, q + 1] for q in range(k)], dtype=np.int64)
    inc = O.incidence(k + 1, edges)
    G0 = rng.normal(size=(2,) + (d,) * k) + 1j * rng.normal(size=(2,) + (d,) * k)
    leaves = [np.eye(2, d, dtype=np.complex128) for _ in range(k)]
    lam = []
    for _ in range(k):
        v = np.sort(rng.random(d))[::-1] + 0.05
        lam.append(v / np.linalg.norm(v))
    st = O.VidalState(k + 1, edges, inc, [G0.astype(np.complex128)] + leaves, lam)
    T = O.symmetric_gauge(st)
    m0 = O.reconstructed_messages(st)
    delta = {}
    for key, v in m0.items():
        A = 0.05 * (rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d)))
        H = A + A.conj().T
        delta[key] = H - np.trace(H) / d * np.eye(d)   # trace-free, Hermitian
    return st, T, m0, delta


@pytest.mark.parametrize("k,d", [(4, 3), (3, 4)])
def test_delta_form_of_the_message_update(k, d):
    st, T, m0, delta = _star(k, d, seed=k * 10 + d)
    m = {key: m0[key] + delta[key] for key in m0}
    centre = 0
    for e_out in st.inc[centre]:
        others = [e for e in st.inc[centre] if e != e_out]
        inward = {e: O.directed(st, st.other(e, centre), e) for e in others}
        F = O.message_update(st, T, m, centre, e_out)
        F0 = O.message_update(st, T, m0, centre, e_out)
        Fd = np.zeros_like(F)
        for c, ec in enumerate(others):
            mix = dict(m0)
            for i, e in enumerate(others):
                key = inward[e]
                mix[key] = m0[key] if i < c else (delta[key] if i == c else m[key])
            Fd = Fd + O.message_update(st, T, mix, centre, e_out)
        assert np.abs(F - (F0 + Fd)).max() < 1e-13 * np.abs(F).max()
        # the normalised update in the delta form
        out = O.directed(st, centre, e_out)
        m0_out = m0[out]
        t0 = np.trace(F0)
        D0 = F0 - t0 * m0_out
        tau = np.trace(Fd)
        dnew = (D0 + Fd - m0_out * tau) / (t0 + tau)
        assert np.abs((F / np.trace(F) - m0_out) - dnew).max() < 1e-13
