"""Exact 2^N statevector simulation of the Trotterised annealing circuit.

TEST INFRASTRUCTURE ONLY (pins for the GTQA oracle; never used by the library).

The circuit is Eq. (discretizatoion) of App. F with reading R1 of the oracle
(layer k applies U_Z(dt*k/K) then U_X(dt*(1-k/K)), k = 1..K), starting from
|+>^N (Sec. III A); `evolve_split` takes any per-layer angles
(t_X_pre, t_Z, t_X_post) (reading R13), and `apply_one` / `apply_two` apply
arbitrary one- and two-qubit gates (reading R14).  U_Z is the product of the commuting diagonal two-qubit gates
exp(-i t (J_ab Z_a Z_b + h_a/D_a Z_a + h_b/D_b Z_b)), U_X the product of
exp(-i t X_a).  Qubit a is tensor axis a; |0> has Z eigenvalue +1 (x_a = +1,
Sec. III A).
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


def plus_state(n: int) -> np.ndarray:
    return np.full((2,) * n, 2.0 ** (-n / 2), dtype=np.complex128)


def z_values(n: int) -> np.ndarray:
    """z[a, x] = +1/-1 for qubit a in basis state x (axis order = qubit order)."""
    idx = np.arange(2 ** n)
    bits = (idx[None, :] >> (n - 1 - np.arange(n))[:, None]) & 1
    return 1 - 2 * bits


def interaction_phase(n: int, edges, J, h) -> np.ndarray:
    """Exponent E(z) of U_Z(t) = exp(-i t E(z)), accumulated gate by gate (App. F)."""
    edges = np.asarray(edges)
    z = z_values(n)
    deg = np.bincount(edges.ravel(), minlength=n)
    E = np.zeros(2 ** n)
    for e, (a, b) in enumerate(edges.tolist()):
        E += J[e] * z[a] * z[b] + h[a] / deg[a] * z[a] + h[b] / deg[b] * z[b]
    return E.reshape((2,) * n)


def apply_mixing(psi: np.ndarray, t: float) -> np.ndarray:
    c, s = np.cos(t), np.sin(t)
    W = np.array([[c, -1j * s], [-1j * s, c]])
    n = psi.ndim
    for a in range(n):
        psi = np.moveaxis(np.tensordot(W, psi, axes=([1], [a])), 0, a)
    return psi


def rdm1(psi: np.ndarray, a: int) -> np.ndarray:
    """Single-qubit reduced density matrix rho_a[i, i']."""
    p = np.moveaxis(psi, a, 0).reshape(2, -1)
    return p @ p.conj().T


def all_rdm1(psi: np.ndarray) -> np.ndarray:
    return np.stack([rdm1(psi, a) for a in range(psi.ndim)])


def schmidt_values(psi: np.ndarray, part_a: Sequence[int]) -> np.ndarray:
    """Schmidt coefficients of psi across the cut (part_a | rest), descending."""
    n = psi.ndim
    part_a = list(part_a)
    rest = [q for q in range(n) if q not in part_a]
    p = np.transpose(psi, part_a + rest).reshape(2 ** len(part_a), -1)
    return np.linalg.svd(p, compute_uv=False)


def evolve(n: int, edges, J, h, K: int, dt: float, layers: int | None = None,
           record: bool = True):
    """Run layers 1..layers (default K).  Returns (psi, [rho per layer])."""
    E = interaction_phase(n, edges, J, h)
    psi = plus_state(n)
    rhos: List[np.ndarray] = []
    last = K if layers is None else layers
    for k in range(1, last + 1):
        tau = k / K
        psi = psi * np.exp(-1j * dt * tau * E)
        psi = apply_mixing(psi, dt * (1.0 - tau))
        if record:
            rhos.append(all_rdm1(psi))
    return psi, rhos


def apply_one(psi: np.ndarray, a: int, W: np.ndarray) -> np.ndarray:
    """psi'[.., i_a, ..] = sum_i' W[i_a, i'] psi[.., i', ..]."""
    return np.moveaxis(np.tensordot(np.asarray(W), psi, axes=([1], [a])), 0, a)


def apply_two(psi: np.ndarray, a: int, b: int, W: np.ndarray) -> np.ndarray:
    """A 4x4 gate W[(i_a i_b), (i_a' i_b')] on qubits a and b."""
    W4 = np.asarray(W).reshape(2, 2, 2, 2)
    out = np.tensordot(W4, psi, axes=([2, 3], [a, b]))
    return np.moveaxis(out, [0, 1], [a, b])


def evolve_split(n: int, edges, J, h, angles, record: bool = True):
    """Layers U_X(t_post) U_Z(t_Z) U_X(t_pre) for each (t_pre, t_Z, t_post) in `angles`.
    Returns (psi, [rho per layer])."""
    E = interaction_phase(n, edges, J, h)
    psi = plus_state(n)
    rhos: List[np.ndarray] = []
    for t_pre, t_Z, t_post in angles:
        if t_pre != 0.0:
            psi = apply_mixing(psi, t_pre)
        psi = psi * np.exp(-1j * t_Z * E)
        if t_post != 0.0:
            psi = apply_mixing(psi, t_post)
        if record:
            rhos.append(all_rdm1(psi))
    return psi, rhos
