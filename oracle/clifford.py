"""Pauli-string propagation through the Clifford circuit U(pi/2) (test infrastructure).

At theta_h = pi/2 every gate of U(theta_h) (Eq. 1) is Clifford, so conjugating
a Pauli string by U(pi/2) gives another Pauli string ("Measuring expectation
values": U^n(pi/2) Z_i U^n(pi/2)^dagger is a single Pauli string, and the paper
prints one example, the weight-10 string from Z_13 after five steps).

Each conjugation is done by brute force on the gate's own qubits: the local
2x2 or 4x4 operator G P G^dagger is formed as a dense matrix and expanded in
the Pauli basis, where exactly one coefficient (a phase in {+-1, +-i}) must be
non-zero.  Nothing relies on symplectic update tables.

Gate conventions (Eq. 1): RX(theta) = exp(-i theta X / 2) acts first, then the
ZZ layer exp(+i pi/4 Z_v Z_w) on every edge; U = (ZZ layer) (RX layer).
"""
from __future__ import annotations

import itertools

import numpy as np

I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
PAULI = {"I": I2, "X": PX, "Y": PY, "Z": PZ}


def rx(theta):
    """exp(-i theta X / 2)."""
    return np.cos(theta / 2) * I2 - 1j * np.sin(theta / 2) * PX


def zz_gate(phi=np.pi / 4):
    """exp(+i phi Z (x) Z) as a 4x4 matrix on (first, second) qubit."""
    zz = np.kron(PZ, PZ)
    return np.cos(phi) * np.eye(4) + 1j * np.sin(phi) * zz


def _decompose(mat, nq):
    """Expand a 2^nq x 2^nq matrix in Pauli products; it must be one term."""
    hits = []
    for labels in itertools.product("IXYZ", repeat=nq):
        p = PAULI[labels[0]]
        for l in labels[1:]:
            p = np.kron(p, PAULI[l])
        coef = np.trace(p.conj().T @ mat) / (2 ** nq)
        if abs(coef) > 1e-9:
            hits.append((labels, coef))
    assert len(hits) == 1, f"not a single Pauli string: {hits}"
    labels, coef = hits[0]
    ph = complex(np.round(coef.real)) + 1j * complex(np.round(coef.imag))
    assert abs(ph - coef) < 1e-9 and abs(abs(ph) - 1) < 1e-12
    return labels, ph


class PauliString:
    """phase * prod_q P_q with P_q in {X, Y, Z} on the listed qubits."""

    def __init__(self, ops=None, phase=1):
        self.ops = {int(q): p for q, p in (ops or {}).items() if p != "I"}
        self.phase = complex(phase)

    def copy(self):
        return PauliString(dict(self.ops), self.phase)

    @property
    def weight(self):
        return len(self.ops)

    def conj_1q(self, q, g):
        """P -> g P g^dagger with g acting on qubit q."""
        p = self.ops.get(q, "I")
        if p == "I":
            return
        labels, ph = _decompose(g @ PAULI[p] @ g.conj().T, 1)
        self.phase *= ph
        if labels[0] == "I":
            self.ops.pop(q)
        else:
            self.ops[q] = labels[0]

    def conj_2q(self, a, b, g):
        """P -> g P g^dagger with g a 4x4 on (a, b), a the first factor."""
        pa, pb = self.ops.get(a, "I"), self.ops.get(b, "I")
        if pa == "I" and pb == "I":
            return
        local = np.kron(PAULI[pa], PAULI[pb])
        labels, ph = _decompose(g @ local @ g.conj().T, 2)
        self.phase *= ph
        for q, l in zip((a, b), labels):
            if l == "I":
                self.ops.pop(q, None)
            else:
                self.ops[q] = l

    def as_tuple(self):
        return tuple(sorted(self.ops.items())), self.phase


def conjugate_by_step(p: PauliString, graph, theta=np.pi / 2) -> PauliString:
    """Return U P U^dagger for one Floquet step U = (ZZ layer)(RX layer)."""
    out = p.copy()
    g1 = rx(theta)
    for q in list(out.ops):
        out.conj_1q(q, g1)
    g2 = zz_gate()
    for (a, b) in graph.edges:
        out.conj_2q(a, b, g2)
    return out


def conjugate_by_step_dagger(p: PauliString, graph, theta=np.pi / 2) -> PauliString:
    """Return U^dagger P U for one Floquet step."""
    out = p.copy()
    g2 = zz_gate().conj().T
    for (a, b) in graph.edges:
        out.conj_2q(a, b, g2)
    g1 = rx(theta).conj().T
    for q in list(out.ops):
        out.conj_1q(q, g1)
    return out


def propagate(p: PauliString, graph, steps, dagger=False, theta=np.pi / 2):
    """U^steps P U^-steps (dagger=False) or U^-steps P U^steps (dagger=True)."""
    out = p.copy()
    for _ in range(steps):
        out = (conjugate_by_step_dagger if dagger else conjugate_by_step)(out, graph, theta)
    return out


def z_string(q):
    return PauliString({q: "Z"})


def expectation_on_zero_state(p: PauliString):
    """<0...0| P |0...0>: phase if P has only Z factors, else 0."""
    if any(l != "Z" for l in p.ops.values()):
        return 0.0
    return p.phase


def clifford_expectation(p: PauliString, graph, steps):
    """<psi(pi/2, steps)| P |psi(pi/2, steps)> by Heisenberg propagation of P."""
    h = propagate(p, graph, steps, dagger=True)
    return expectation_on_zero_state(h)


def string_from_z(graph, site, nprime):
    """The Pauli string U^n'(pi/2) Z_site U^n'(pi/2)^dagger ("extended time
    evolution" identity).  Returns a PauliString (phase is +-1)."""
    return propagate(z_string(site), graph, nprime, dagger=False)


def parse_string(spec: str) -> PauliString:
    """Parse e.g. 'X13,29,31 Y9,30 Z8,12,17,28,32' into a PauliString."""
    ops = {}
    for tok in spec.split():
        lab, qs = tok[0], tok[1:]
        for q in qs.split(","):
            ops[int(q)] = lab
    return PauliString(ops)
