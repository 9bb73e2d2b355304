"""The BP-approximated tensor-network state algorithm in FP64 (test infrastructure).

This is the method of the paper (Tindall et al., arXiv:2306.14887) written out
step by step in NumPy complex128, for checking the library against.  It is an
approximation (truncated simple update with belief-propagation environments),
so the oracle is the algorithm itself in the paper's order:

* State ("State ansatz", Fig. "heavyhexdiagram"): one tensor T_v[p, l_1..l_d]
  per qubit, physical index p first, then one virtual leg per incident edge in
  increasing edge id.  The state is kept in an arbitrary gauge together with
  BP messages, which the Methods section states gives the same results as the
  Vidal gauge (section "The Vidal gauge", last paragraph).
* Initial state |0...0> ("State ansatz"): every bond of dimension 1.
* One Floquet step U(theta_h) (Eq. 1): RX(theta_h) = exp(-i theta_h X/2) on
  every qubit, applied exactly; then exp(+i pi/4 Z_v Z_w) on every edge, by
  simple update ("The simple update procedure", Fig. "SimpleUpdate") in the
  message formulation: the environment of each tensor is the product of its
  incoming messages, the gate bond is truncated back to chi by an SVD, and
  the message on the gate edge is replaced by the new bond matrix diag(S).
  Edges are applied in colour layers 0, 1, 2 (disjoint edges within a layer).
* After each step the network is regauged by belief propagation ("State
  ansatz": regauging after every Trotter step), iterating Eq.
  "MessageTensorSelfConsistency" with the norm tensor kept as T and T* (Eq.
  "SymmetricTensor" and the sentence after it).
* Expectation values ("Measuring expectation values", Eqs. "SingleSIte",
  "SquareBondTensors"): rho_v from T_v, T_v* and the incoming messages.
  Pauli strings either by exact contraction over a tree spanning the string
  with BP messages on every other edge, or by the extended time evolution
  identity (U^n'(pi/2) Z_i U^n'(pi/2)^dagger is a single Pauli string).

Readings where the paper is silent (each listed in the project's design notes):
message index order M[ket, bra]; synchronous BP sweeps warm-started from the
current messages; messages Hermitised and scaled to unit Frobenius norm;
convergence when max ||M_new - M_old||_F < tol; truncation keeps the chi
largest singular values (those above 1e-13 sigma_1) and renormalises
||S||_2 = 1; sqrt(S) goes to each side; environment square roots use the
Hermitian square root of each message with eigenvalues below 1e-14 lambda_max
dropped (pseudo-inverse on the un-absorb); the gate is split as
exp(i pi/4 ZZ) = sum_k A_k (x) B_k with A_0 = B_0 = 2^-1/4 I,
A_1 = 2^-1/4 Z, B_1 = i 2^-1/4 Z.
"""
from __future__ import annotations

import numpy as np

from . import clifford as C

EIG_CUTOFF = 1e-14
SVD_CUTOFF = 1e-13


def rx(theta):
    """exp(-i theta X / 2) (Eq. 1)."""
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    return np.array([[c, -1j * s], [-1j * s, c]])


def gate_split(sign=+1):
    """Operator-Schmidt factors of exp(sign * i pi/4 Z(x)Z) as diagonals a_k, b_k.

    exp(i phi ZZ) = cos(phi) I(x)I + i sin(phi) Z(x)Z; at phi = pi/4 both weights
    are 1/sqrt(2), split evenly between the two sides."""
    r = 2.0 ** -0.25
    z = np.array([1.0, -1.0])
    a = np.array([[r, r], r * z], dtype=complex)
    b = np.array([[r, r], sign * 1j * r * z], dtype=complex)
    return a, b


class BPState:
    """Site tensors, directed BP messages and bond dimensions for a graph."""

    def __init__(self, graph, chi):
        self.g = graph
        self.chi = int(chi)
        self.T = []
        for v in range(graph.n):
            t = np.zeros((2,) + (1,) * graph.degree(v), dtype=complex)
            t[(0,) * (1 + graph.degree(v))] = 1.0
            self.T.append(t)
        # message from src across edge e: key (src, e); shape (d_e, d_e), [ket, bra]
        self.M = {}
        for e, (u, w) in enumerate(graph.edges):
            self.M[(u, e)] = np.ones((1, 1), dtype=complex)
            self.M[(w, e)] = np.ones((1, 1), dtype=complex)
        self.discarded = []        # discarded weight per applied gate
        self.min_gap = np.inf      # smallest relative gap at a truncation

    # ------------------------------------------------------------------ utils
    def leg_pos(self, v, e):
        return 1 + self.g.legs[v].index(e)

    def incoming(self, v, e):
        """Message into v along edge e (sent by the other endpoint)."""
        return self.M[(self.g.other(e, v), e)]

    def dim(self, e):
        u = self.g.edges[e][0]
        return self.T[u].shape[self.leg_pos(u, e)]

    def copy(self):
        out = BPState.__new__(BPState)
        out.g, out.chi = self.g, self.chi
        out.T = [t.copy() for t in self.T]
        out.M = {k: m.copy() for k, m in self.M.items()}
        out.discarded = list(self.discarded)
        out.min_gap = self.min_gap
        return out

    # ------------------------------------------------------ single-site gate
    def apply_1q(self, u):
        """T_v <- u applied on the physical leg of every site."""
        self.T = [np.tensordot(u, t, axes=(1, 0)) for t in self.T]

    def apply_rx(self, theta):
        self.apply_1q(rx(theta))

    # ----------------------------------------------------------- BP messages
    def _contract_except(self, v, skip):
        """T_v with every leg except ``skip`` contracted (ket side) against the
        incoming message: result index order unchanged, leg x now carries the
        bra index of M_x."""
        x = self.T[v]
        for e in self.g.legs[v]:
            if e == skip:
                continue
            ax = self.leg_pos(v, e)
            m = self.incoming(v, e)
            x = np.moveaxis(np.tensordot(x, m, axes=(ax, 0)), -1, ax)
        return x

    def message(self, v, e):
        """Eq. "MessageTensorSelfConsistency": M_{v -> w}[e, e'] =
        sum T_v[p, .., e, ..] conj(T_v[p, .., e', ..]) prod_{x != e} M_{x -> v}."""
        x = self._contract_except(v, e)
        ax = self.leg_pos(v, e)
        others = [i for i in range(x.ndim) if i != ax]
        return np.tensordot(x, np.conj(self.T[v]), axes=(others, others))

    @staticmethod
    def normalise(m):
        """Hermitise and scale to unit Frobenius norm."""
        m = 0.5 * (m + m.conj().T)
        return m / np.linalg.norm(m)

    def bp_sweep(self):
        """One synchronous sweep over every directed edge; returns the residual
        max ||M_new - M_old||_F (messages compared after normalisation)."""
        new = {}
        for (src, e) in self.M:
            new[(src, e)] = self.normalise(self.message(src, e))
        res = max(np.linalg.norm(new[k] - self.M[k]) for k in new)
        self.M = new
        return res

    def bp_converge(self, tol=1e-10, max_iters=1000):
        for it in range(1, max_iters + 1):
            res = self.bp_sweep()
            if res < tol:
                return it, res
        return max_iters, res

    # ------------------------------------------------------- simple update
    @staticmethod
    def _sqrt_pair(m):
        """Hermitian square root B of a PSD message and its pseudo-inverse."""
        m = 0.5 * (m + m.conj().T)
        lam, w = np.linalg.eigh(m)
        keep = lam > EIG_CUTOFF * max(lam.max(), 0.0)
        r = np.where(keep, np.sqrt(np.where(keep, lam, 0.0)), 0.0)
        ri = np.where(keep, 1.0 / np.where(keep, r, 1.0), 0.0)
        return (w * r) @ w.conj().T, (w * ri) @ w.conj().T

    def _absorbed_matrix(self, v, e, coef):
        """Absorb B_x = sqrt(M_{x->v}) on every leg x != e, then reshape to a
        matrix with rows (p, other legs) and columns (e, k) where column block k
        is the gate-split factor coef[k][p] times the absorbed tensor."""
        x = self.T[v]
        inv = {}
        for f in self.g.legs[v]:
            if f == e:
                continue
            b, binv = self._sqrt_pair(self.incoming(v, f))
            inv[f] = binv
            ax = self.leg_pos(v, f)
            x = np.moveaxis(np.tensordot(x, b, axes=(ax, 0)), -1, ax)
        ax = self.leg_pos(v, e)
        x = np.moveaxis(x, ax, -1)                 # (p, others..., e)
        shape = x.shape
        mat = x.reshape(2, -1, shape[-1])          # (p, rows, e)
        blocks = [(coef[k][:, None, None] * mat).reshape(-1, shape[-1]) for k in range(2)]
        return np.concatenate(blocks, axis=1), shape, inv

    def _restore(self, v, e, mat, shape, inv):
        """Inverse of _absorbed_matrix for the new bond: reshape, move the bond
        back to its leg position, and apply the pseudo-inverse square roots."""
        x = mat.reshape(shape[:-1] + (mat.shape[1],))
        x = np.moveaxis(x, -1, self.leg_pos(v, e))
        for f, binv in inv.items():
            ax = self.leg_pos(v, f)
            x = np.moveaxis(np.tensordot(x, binv, axes=(ax, 0)), -1, ax)
        return x

    def apply_zz(self, e, sign=+1):
        """Simple update of exp(sign * i pi/4 Z_v Z_w) on edge e (v = lower id)."""
        v, w = self.g.edges[e]
        a, b = gate_split(sign)
        xv, shv, invv = self._absorbed_matrix(v, e, a)
        xw, shw, invw = self._absorbed_matrix(w, e, b)
        qv, rv = np.linalg.qr(xv)
        qw, rw = np.linalg.qr(xw)
        u, s, vh = np.linalg.svd(rv @ rw.T)
        nz = int(np.sum(s > SVD_CUTOFF * s[0])) if s[0] > 0 else 1
        keep = max(1, min(self.chi, nz))
        total = np.sum(s ** 2)
        self.discarded.append(float(np.sum(s[keep:] ** 2) / total))
        if keep < nz:
            self.min_gap = min(self.min_gap, float((s[keep - 1] - s[keep]) / s[0]))
        sk = s[:keep] / np.linalg.norm(s[:keep])
        left = (qv @ u[:, :keep]) * np.sqrt(sk)
        right = (qw @ vh[:keep, :].T) * np.sqrt(sk)
        self.T[v] = self._restore(v, e, left, shv, invv)
        self.T[w] = self._restore(w, e, right, shw, invw)
        m = np.diag(sk).astype(complex)
        self.M[(v, e)] = m.copy()
        self.M[(w, e)] = m.copy()

    def zz_layers(self, sign=+1):
        for layer in self.g.layers():
            for e in layer:
                self.apply_zz(e, sign)

    # ------------------------------------------------------------- Floquet
    def floquet_step(self, theta, tol=1e-10, max_iters=1000):
        """One application of U(theta_h) (Eq. 1), then BP regauge."""
        self.apply_rx(theta)
        self.zz_layers(+1)
        return self.bp_converge(tol, max_iters)

    def clifford_dagger_step(self, tol=1e-10, max_iters=1000):
        """One application of U(pi/2)^dagger: ZZ^dagger layers, then RX(-pi/2)."""
        self.zz_layers(-1)
        self.apply_rx(-np.pi / 2)
        return self.bp_converge(tol, max_iters)

    # ---------------------------------------------------------- expectations
    def rho(self, v):
        """rho_v[p, p'] = sum T_v[p, ..] conj(T_v[p', ..]) prod_x M_{x->v}."""
        x = self._contract_except(v, None)
        axes = list(range(1, x.ndim))
        return np.tensordot(x, np.conj(self.T[v]), axes=(axes, axes))

    def expect_1q(self, v, op):
        r = self.rho(v)
        return complex(np.trace(r @ op) / np.trace(r))

    def expect_z(self, v):
        r = self.rho(v)
        return float(((r[0, 0] - r[1, 1]) / (r[0, 0] + r[1, 1])).real)

    def all_z(self):
        return np.array([self.expect_z(v) for v in range(self.g.n)])

    def region_expectation(self, ops, phase=1.0):
        """Pauli string by exact contraction over a tree spanning its support,
        every other edge closed by the converged messages."""
        tree_edges = steiner_tree(self.g, sorted(ops))
        verts = sorted({x for e in tree_edges for x in self.g.edges[e]} | set(ops))
        num = self._tree_contract(verts, tree_edges, ops)
        den = self._tree_contract(verts, tree_edges, {})
        return complex(phase * num / den)

    def _tree_contract(self, verts, tree_edges, ops):
        tset = set(tree_edges)
        adj = {v: [e for e in self.g.legs[v] if e in tset] for v in verts}
        root = verts[0]
        order, parent = [], {root: None}
        stack = [root]
        while stack:                      # DFS preorder
            v = stack.pop()
            order.append(v)
            for e in adj[v]:
                w = self.g.other(e, v)
                if w not in parent:
                    parent[w] = e
                    stack.append(w)
        up = {}
        for v in reversed(order):
            x = self.T[v]
            o = C.PAULI[ops.get(v, "I")]
            # insert the operator: sum_p' O[p', p] ... conj(T[p', ..])
            tb = np.tensordot(o.T, np.conj(self.T[v]), axes=(1, 0))
            for e in self.g.legs[v]:
                if e == parent[v]:
                    continue
                ax = self.leg_pos(v, e)
                if e in tset:
                    m = up[(self.g.other(e, v), e)]
                else:
                    m = self.incoming(v, e)
                x = np.moveaxis(np.tensordot(x, m, axes=(ax, 0)), -1, ax)
            if parent[v] is None:
                axes = list(range(x.ndim))
                return complex(np.tensordot(x, tb, axes=(axes, axes)))
            ax = self.leg_pos(v, parent[v])
            others = [i for i in range(x.ndim) if i != ax]
            up[(v, parent[v])] = np.tensordot(x, tb, axes=(others, others))
        raise AssertionError("unreachable")


def steiner_tree(g, terminals):
    """Edges of a tree spanning the terminals: union of BFS shortest paths from
    the first terminal (deterministic, lowest-id tie-breaking), then pruned of
    non-terminal leaves."""
    from collections import deque
    if len(terminals) <= 1:
        return []
    src = terminals[0]
    par = {src: None}
    q = deque([src])
    while q:
        v = q.popleft()
        for e in g.legs[v]:
            w = g.other(e, v)
            if w not in par:
                par[w] = e
                q.append(w)
    edges = set()
    for t in terminals[1:]:
        v = t
        while par[v] is not None:
            edges.add(par[v])
            v = g.other(par[v], v)
    return sorted(edges)


def run(graph, chi, theta, steps, tol=1e-10, max_iters=1000, record=None):
    """Evolve |0...0> by ``steps`` Floquet steps; returns the final BPState.
    ``record(step, state, iters, residual)`` is called after each step."""
    st = BPState(graph, chi)
    for s in range(steps):
        it, res = st.floquet_step(theta, tol, max_iters)
        if record is not None:
            record(s + 1, st, it, res)
    return st


def extended_string_expectation(state, site, nprime, tol=1e-10, max_iters=1000):
    """<psi| S |psi> for the string S = U^n'(pi/2) Z_site U^n'(pi/2)^dagger / phase
    by further evolving with U(pi/2)^dagger n' times and measuring Z_site
    ("Measuring expectation values").  Returns (value, PauliString)."""
    s = C.string_from_z(state.g, site, nprime)
    st = state.copy()
    for _ in range(nprime):
        st.clifford_dagger_step(tol, max_iters)
    return st.expect_z(site) / s.phase.real, s
