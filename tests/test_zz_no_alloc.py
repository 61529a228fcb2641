"""BP entry point that allocates no device memory (gtqa_bp_static).

It exists for callers that cannot call cudaMalloc from this code path (allocation-free
latency-bound loops, or processes whose device memory belongs to another allocator).
Its scratch is a file-scope device array shared by every call, so this file is
collected last and checks two calls in a row against the allocating entry point.
"""
import numpy as np
import pytest

import gpu_util as U
from instances import make_instance
from oracle import gtqa_oracle as O

pytestmark = pytest.mark.gpu


def _graph_arrays(inst):
    """vert_edges [n][4] (slot edges, degree) and edge_info [m][4] (u, v, slots)."""
    inc = O.incidence(inst.n, inst.edges)
    ve = np.full((inst.n, 4), -1, dtype=np.int32)
    for a in range(inst.n):
        for k, e in enumerate(inc[a]):
            ve[a, k] = e
        ve[a, 3] = len(inc[a])
    ei = np.zeros((inst.m, 4), dtype=np.int32)
    for e, (u, v) in enumerate(inst.edges.tolist()):
        ei[e] = (u, v, inc[u].index(e), inc[v].index(e))
    return ve, ei


def test_static_bp_matches_allocating_bp_twice():
    torch = pytest.importorskip("torch")
    G = U.lib()
    inst = make_instance(16, 3)
    s = G.gtqa_create(inst.n, inst.edges, inst.J, inst.h, 4, inst.colour)
    try:
        for k in range(1, 7):
            G.gtqa_trotter_layer(s, k / 20, 0.1)
            G.gtqa_bp_sweep(s, 1e-12, 100)
        G.gtqa_trotter_layer(s, 7 / 20, 0.1)
        Gm, L, _ = G.gtqa_get_state(s)
        it_ref, d_ref, _ = G.gtqa_bp_sweep(s, 1e-12, 100, G.GTQA_BP_WARM_START)
        _, _, M_ref = G.gtqa_get_state(s)
    finally:
        G.gtqa_destroy(s)
    ve, ei = _graph_arrays(inst)
    dev = torch.device("cuda")
    d_ve = torch.from_numpy(ve).to(dev)
    d_ei = torch.from_numpy(ei).to(dev)
    d_g = torch.from_numpy(Gm).to(dev)
    d_l = torch.from_numpy(L).to(dev)
    # the oracle's flooding BP (App. B) from the same state and warm start
    st = O.from_padded(inst.n, inst.edges, Gm, L)
    T = O.symmetric_gauge(st)
    msgs, it_o, hist = O.bp(st, T, O.reconstructed_messages(st), 1e-12, 100)
    M_ora = O.messages_to_padded(st, msgs, 4)
    for call in range(2):
        out = torch.full((2 * inst.m, 4, 4), complex(np.nan, np.nan), dtype=torch.complex128, device=dev)
        rc, it, d = G.gtqa_bp_static(inst.n, inst.m, d_ve, d_ei, d_g, d_l, out, 1e-12, 100)
        torch.cuda.synchronize()
        M = out.cpu().numpy()
        assert rc == G.GTQA_OK and it == it_ref, (call, rc, it, it_ref)
        assert abs(d - d_ref) <= 1e-10 * max(1.0, abs(d_ref))
        assert np.abs(M - M_ref).max() < 1e-10, call
        assert abs(it - it_o) <= 1 and abs(d - hist[-1]) < 1e-10, (it, it_o, d, hist[-1])
        assert np.abs(M - M_ora).max() < 1e-10, call


def test_static_bp_rejects_oversize_and_host_pointers():
    torch = pytest.importorskip("torch")
    G = U.lib()
    dev = torch.device("cuda")
    buf = torch.zeros(16, dtype=torch.float64, device=dev)
    with pytest.raises(G.GTQAError) as ei:
        G.gtqa_bp_static(4096, 10, buf, buf, buf, buf, buf, 1e-8, 10)
    assert ei.value.code == G.GTQA_ERR_INVALID_ARG
    host = np.zeros(16)
    with pytest.raises(G.GTQAError) as ei:
        G.gtqa_bp_static(4, 4, host, host, host, host, host, 1e-8, 10)
    assert ei.value.code == G.GTQA_ERR_INVALID_ARG


def test_static_bp_rejects_inconsistent_index_arrays():
    """The index arrays are checked on the device before BP reads through them: an edge id
    out of range, a degree above 3 or slots that disagree between the two arrays return
    GTQA_ERR_INVALID_ARG, and a later call with the correct arrays still works."""
    torch = pytest.importorskip("torch")
    G = U.lib()
    inst = make_instance(16, 3)
    ve, ei = _graph_arrays(inst)
    dev = torch.device("cuda")
    Gm = np.zeros((inst.n, 2, 4, 4, 4), dtype=np.complex128)
    Gm[:, :, 0, 0, 0] = 1.0 / np.sqrt(2.0)
    L = np.zeros((inst.m, 4))
    L[:, 0] = 1.0
    d_g = torch.from_numpy(Gm).to(dev)
    d_l = torch.from_numpy(L).to(dev)
    out = torch.zeros((2 * inst.m, 4, 4), dtype=torch.complex128, device=dev)
    bad_cases = []
    v = ve.copy(); v[3, 1] = inst.m + 5; bad_cases.append((v, ei))          # edge id out of range
    v = ve.copy(); v[0, 3] = 4; bad_cases.append((v, ei))                   # degree above 3
    e = ei.copy(); e[2, 2] = (e[2, 2] + 1) % 3; bad_cases.append((ve, e))   # slot that names another edge
    e = ei.copy(); e[5, 0] = -1; bad_cases.append((ve, e))                  # endpoint out of range
    for v, e in bad_cases:
        with pytest.raises(G.GTQAError) as err:
            G.gtqa_bp_static(inst.n, inst.m, torch.from_numpy(v).to(dev), torch.from_numpy(e).to(dev), d_g, d_l,
                             out, 1e-12, 10)
        assert err.value.code == G.GTQA_ERR_INVALID_ARG
    rc, it, d = G.gtqa_bp_static(inst.n, inst.m, torch.from_numpy(ve).to(dev), torch.from_numpy(ei).to(dev), d_g,
                                 d_l, out, 1e-12, 10)
    assert rc == G.GTQA_OK and it == 1 and d < 1e-12
