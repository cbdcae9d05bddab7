"""Brute-force Jordan-Wigner state vector (n <= 16 modes).

TEST INFRASTRUCTURE ONLY: an independent checker for the oracle. It applies
each gate of the circuit to the full 2^n-amplitude qubit state and never forms
a mode-transformation matrix, a determinant or a branch sum.

Qubit m holds the occupation of fermionic mode m. With the Jordan-Wigner
mapping a nearest-neighbour hopping a_p^dag a_{p+1} carries no parity string,
so a Givens rotation on modes (p, p+1) is the 2-qubit gate that acts as its
2x2 single-particle matrix g on the one-particle states {|1_p 0_q>, |0_p 1_q>}
(column convention: the state with mode p occupied goes to
g[p,p] |1_p 0_q> + g[q,p] |0_p 1_q>), multiplies |1_p 1_q> by det g and leaves
|0_p 0_q> alone. PHASE multiplies the amplitudes with mode p occupied by
e^{i phi}; CPHASE multiplies those with both p and q occupied by e^{i theta}
(Section II-B: particle-number-conserving matchgates; Eq. 7's left-hand side).
"""
from __future__ import annotations

import math

import numpy as np

GIVENS, PHASE, CPHASE = 0, 1, 2


def _givens_2x2(theta: float, phi: float) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, -np.exp(1j * phi) * s], [np.exp(-1j * phi) * s, c]], dtype=np.complex128)


def run_statevector(n_modes: int, occupation_modes, gates) -> np.ndarray:
    """Final state vector (length 2^n) of the circuit applied to the basis
    state with the given occupied modes."""
    if n_modes > 16:
        raise ValueError("brute-force state vector limited to 16 modes")
    dim = 1 << n_modes
    idx = np.arange(dim, dtype=np.int64)
    psi = np.zeros(dim, dtype=np.complex128)
    a = 0
    for m in occupation_modes:
        a |= 1 << m
    psi[a] = 1.0
    for g in gates:
        kind, p, q = int(g["kind"]), int(g["p"]), int(g["q"])
        if kind == GIVENS:
            G = _givens_2x2(float(g["theta"]), float(g["phi"]))
            np_ = (idx >> p) & 1
            nq = (idx >> q) & 1
            s10 = idx[(np_ == 1) & (nq == 0)]  # mode p occupied, q empty
            s01 = s10 ^ (1 << p) ^ (1 << q)    # partner: mode q occupied, p empty
            v10, v01 = psi[s10].copy(), psi[s01].copy()
            psi[s10] = G[0, 0] * v10 + G[0, 1] * v01
            psi[s01] = G[1, 0] * v10 + G[1, 1] * v01
            s11 = idx[(np_ == 1) & (nq == 1)]
            psi[s11] *= G[0, 0] * G[1, 1] - G[0, 1] * G[1, 0]
        elif kind == PHASE:
            sel = ((idx >> p) & 1) == 1
            psi[sel] *= np.exp(1j * float(g["phi"]))
        elif kind == CPHASE:
            sel = (((idx >> p) & 1) == 1) & (((idx >> q) & 1) == 1)
            psi[sel] *= np.exp(1j * float(g["theta"]))
        else:
            raise ValueError(f"unknown gate kind {kind}")
    return psi


def amplitudes(n_modes: int, occupation_modes, gates, bitstrings_modes) -> np.ndarray:
    psi = run_statevector(n_modes, occupation_modes, gates)
    out = np.empty(len(bitstrings_modes), dtype=np.complex128)
    for i, modes in enumerate(bitstrings_modes):
        b = 0
        for m in modes:
            b |= 1 << m
        out[i] = psi[b]
    return out
