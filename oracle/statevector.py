"""O2: dense FP64 state-vector simulator -- test infrastructure only.

The quantity it computes is the plain definition of an output amplitude,
a_x = <x| C |0...0>, where C is the circuit (the state |psi> of the paper's
PEPS equation, written out in the computational basis instead of as a PEPS).

Conventions: the state is a complex128 vector of length 2^n; bit q of the
index is the value of qubit q (q = r*C + c on the lattice).
"""
from __future__ import annotations

import numpy as np


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def apply_1q(psi: np.ndarray, n: int, q: int, U: np.ndarray) -> None:
    """psi <- (U acting on qubit q) psi, in place.  U[out, in]."""
    v = psi.reshape(1 << (n - q - 1), 2, 1 << q)
    a0 = v[:, 0, :].copy()
    a1 = v[:, 1, :].copy()
    v[:, 0, :] = U[0, 0] * a0 + U[0, 1] * a1
    v[:, 1, :] = U[1, 0] * a0 + U[1, 1] * a1


def apply_cz(psi: np.ndarray, n: int, q0: int, q1: int) -> None:
    """psi <- CZ(q0, q1) psi in place: the sign of every basis state with both
    bits set flips."""
    lo, hi = min(q0, q1), max(q0, q1)
    v = psi.reshape(1 << (n - hi - 1), 2, 1 << (hi - lo - 1), 2, 1 << lo)
    v[:, 1, :, 1, :] *= -1.0


def apply_2q(psi: np.ndarray, n: int, q0: int, q1: int, G: np.ndarray) -> None:
    """psi <- (G acting on qubits q0, q1) psi in place; G[(t0 t1), (s0 s1)]
    with qubit q0's bit first."""
    G4 = np.asarray(G, dtype=np.complex128).reshape(2, 2, 2, 2)
    v = psi.reshape([2] * n)                 # axis n-1-q holds bit q
    a0, a1 = n - 1 - q0, n - 1 - q1
    w = np.tensordot(G4, v, axes=([2, 3], [a0, a1]))   # new axes 0, 1 = t0, t1
    psi[:] = np.moveaxis(w, [0, 1], [a0, a1]).reshape(-1)


def run(n: int, gates) -> np.ndarray:
    """Final state of the gate list (objects with .kind, .qubits, .U)."""
    if n > 25:
        raise ValueError("state vector limited to 25 qubits")
    psi = zero_state(n)
    for g in gates:
        if g.kind == "1q":
            apply_1q(psi, n, g.qubits[0], np.asarray(g.U, dtype=np.complex128))
        elif g.kind == "cz":
            apply_cz(psi, n, g.qubits[0], g.qubits[1])
        elif g.kind == "2q":
            apply_2q(psi, n, g.qubits[0], g.qubits[1], g.U)
        else:
            raise ValueError(f"unknown gate kind {g.kind}")
    return psi


def amplitudes(n: int, gates, bitstrings) -> np.ndarray:
    psi = run(n, gates)
    idx = np.asarray(bitstrings, dtype=np.uint64).astype(np.int64)
    return psi[idx]


def marginals(n: int, gates, bitstrings, mask: int) -> np.ndarray:
    """Marginal probabilities P(x_S) = sum over the unmeasured bits of |psi_x|^2
    (the definition), for the measured set S = the set bits of `mask`; the
    values of the measured bits are taken from each bitstring."""
    psi = run(n, gates)
    prob = np.abs(psi) ** 2
    idx = np.arange(1 << n, dtype=np.int64)
    out = np.empty(len(bitstrings))
    for i, x in enumerate(bitstrings):
        out[i] = prob[(idx & mask) == (int(x) & mask)].sum()
    return out
