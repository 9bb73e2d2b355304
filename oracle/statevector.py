"""Exact statevector references (test infrastructure; see ``oracle/__init__``).

``evolve`` applies the Floquet unitary of Eq. 1 literally to the initial
state |0...0> (all spins up, "State ansatz"): per step, RX(theta) =
exp(-i theta X/2) on every qubit, then exp(+i pi/4 Z_v Z_w) on every edge.
Qubit q is bit q of the amplitude index.  Usable up to ~22 qubits.

``lightcone_expectation`` gives the exact value of a Pauli string on a large
graph after n steps by simulating only the ball of radius n-1 around the
string's support, with every gate whose qubits lie in that ball.  This is
exact: in the Heisenberg picture the support of U^-n P U^n grows by one graph
step per ZZ layer, starting from supp(P) after the last step, so it stays
inside the ball, and every gate touching it has both ends inside the ball;
the extra gates inside the ball act outside the operator's current support
and commute with it.  The paper quotes such "brute force light cone" results
as the exact reference for 127 qubits after 5 steps ("Results").
"""
from __future__ import annotations

import numpy as np

from . import graph as G


def _apply_1q(psi, n, q, u):
    v = psi.reshape(2 ** (n - q - 1), 2, 2 ** q)
    out = np.einsum("ab,ibj->iaj", u, v)
    return out.reshape(-1)


def _spins(n):
    idx = np.arange(2 ** n, dtype=np.int64)
    return [(1 - 2 * ((idx >> q) & 1)).astype(np.int8) for q in range(n)]


def zz_layer_phase(n, edges):
    """Diagonal of prod_edges exp(+i pi/4 Z_a Z_b) over all basis states."""
    s = _spins(n)
    acc = np.zeros(2 ** n, dtype=np.int64)
    for a, b in edges:
        acc += s[a].astype(np.int64) * s[b]
    return np.exp(1j * np.pi / 4 * acc)


def rx(theta):
    return np.array([[np.cos(theta / 2), -1j * np.sin(theta / 2)],
                     [-1j * np.sin(theta / 2), np.cos(theta / 2)]])


def evolve(graph, theta, steps, psi=None, record=None):
    """|psi(theta, steps)> = U^steps |0...0>; ``record(step, psi)`` per step."""
    n = graph.n
    if psi is None:
        psi = np.zeros(2 ** n, dtype=complex)
        psi[0] = 1.0
    phase = zz_layer_phase(n, graph.edges)
    u = rx(theta)
    for s in range(steps):
        for q in range(n):
            psi = _apply_1q(psi, n, q, u)
        psi = psi * phase
        if record is not None:
            record(s + 1, psi)
    return psi


def evolve_dagger_clifford(graph, psi, steps):
    """Apply (U(pi/2)^dagger)^steps: ZZ^dagger layer, then RX(-pi/2) per step."""
    n = graph.n
    phase = np.conj(zz_layer_phase(n, graph.edges))
    u = rx(-np.pi / 2)
    for _ in range(steps):
        psi = psi * phase
        for q in range(n):
            psi = _apply_1q(psi, n, q, u)
    return psi


def z_expectations(psi, n):
    p = np.abs(psi) ** 2
    idx = np.arange(2 ** n, dtype=np.int64)
    return np.array([np.sum(p * (1 - 2 * ((idx >> q) & 1))) for q in range(n)])


_PM = {"X": np.array([[0, 1], [1, 0]], dtype=complex),
       "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
       "Z": np.array([[1, 0], [0, -1]], dtype=complex)}


def pauli_expectation(psi, n, ops, phase=1.0):
    """<psi| phase * prod_q P_q |psi> for ops = {qubit: 'X'|'Y'|'Z'}."""
    phi = psi
    for q, l in ops.items():
        phi = _apply_1q(phi, n, q, _PM[l])
    return complex(phase * np.vdot(psi, phi))


def lightcone_expectation(graph, theta, steps, ops, phase=1.0):
    """Exact <psi(theta, steps)| P |psi(theta, steps)> on a large graph."""
    assert steps >= 1
    region = graph.ball(list(ops), steps - 1)
    sub = G.induced(graph, region)
    rel = {v: i for i, v in enumerate(region)}
    psi = evolve(sub, theta, steps)
    return pauli_expectation(psi, sub.n, {rel[q]: l for q, l in ops.items()}, phase)


def lightcone_size(graph, sites, steps):
    return len(graph.ball(list(sites), steps - 1))
