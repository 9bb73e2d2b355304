"""Pins of the CPU oracle against facts fixed by the paper or by mathematics.

Nothing here compares the oracle with itself: each check is a printed value
(the weight-10 string), a closed form (the Clifford points), a textbook
construction (dense Kronecker-product unitaries), an exactness statement of
the paper (BP exact on trees and for circuits shorter than the loop length)
or an invariant of the definitions (Hermitian unit-norm messages, gauge
invariance).
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import bptn as B
from oracle import clifford as C
from oracle import graph as G
from oracle import statevector as S
from workloads import random_psd, rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- lattice
def test_eagle_counts():
    """Fig. "heavyhexdiagram": 6 x 3 heavy hexagons plus qubits 13 and 113."""
    g = G.eagle127()
    assert g.n == 127 and len(g.edges) == 144
    hist = G.degree_histogram(g)
    assert list(hist) == [0, 2, 89, 36]
    assert [v for v in range(g.n) if g.degree(v) == 1] == [13, 113]
    # no two degree-3 vertices are adjacent (every edge carries a heavy-hex bridge)
    assert all(not (g.degree(u) == 3 and g.degree(w) == 3) for u, w in g.edges)
    assert g.colouring_is_proper()
    assert [len(l) for l in g.layers()] == [51, 48, 45]


@pytest.mark.parametrize("R,L,n,m", [(5, 11, 65, 72), (13, 27, 433, 504), (21, 43, 1121, 1320)])
def test_heavy_hex_sizes(R, L, n, m):
    g = G.heavy_hex(R, L)
    assert (g.n, len(g.edges)) == (n, m)
    assert g.colouring_is_proper()
    assert max(g.degree(v) for v in range(g.n)) == 3


def test_hexagon_patch_is_a_ring():
    one, two = G.hexagon_patches()
    assert one.n == 12 and len(one.edges) == 12
    assert all(one.degree(v) == 2 for v in range(12))
    assert two.n == 21 and len(two.edges) == 22


def test_lightcone_ball_sizes():
    """The largest backward light cone (ball of radius n-1) on 127 qubits."""
    g = G.eagle127()
    got = [max(len(g.ball([v], n - 1)) for v in range(g.n)) for n in (4, 5, 6)]
    assert got == [13, 19, 31]


# --------------------------------------------------------- Clifford string
def _golden_string():
    spec = {}
    for line in open(os.path.join(GOLDEN, "eagle127_weight10_string.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split(None, 1)
        spec[k] = v.strip()
    return int(spec["site"]), int(spec["nprime"]), int(spec["sign"]), C.parse_string(spec["string"])


def test_printed_weight10_string():
    """X_{13,29,31} Y_{9,30} Z_{8,12,17,28,32} = U^5(pi/2) Z_13 U^5(pi/2)^dagger."""
    site, nprime, sign, want = _golden_string()
    got = C.string_from_z(G.eagle127(), site, nprime)
    assert got.ops == want.ops
    assert got.phase == sign
    assert got.weight == 10


def test_reverse_ordering_differs():
    """U^-5 Z_13 U^5 is a different string: the printed one fixes the order."""
    _, _, _, want = _golden_string()
    other = C.propagate(C.z_string(13), G.eagle127(), 5, dagger=True)
    assert other.ops != want.ops


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_clifford_point_z_vanishes(n):
    """At theta_h = pi/2 every <Z_v> is 0 for n >= 1 (exact Clifford values)."""
    g = G.eagle127()
    for v in (0, 13, 40, 62, 113, 126):
        assert C.clifford_expectation(C.z_string(v), g, n) == 0.0


# ----------------------------------------------------------- statevector
def _dense_unitary(graph, theta):
    """U(theta) of Eq. 1 as a dense matrix from Hamiltonian exponentials."""
    n = graph.n
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Z = np.diag([1.0, -1.0]).astype(complex)

    def embed(ops):
        # qubit q is bit q of the index: kron order is (q = n-1, ..., 0)
        m = np.eye(1)
        for q in reversed(range(n)):
            m = np.kron(m, ops.get(q, np.eye(2)))
        return m

    u = np.eye(2 ** n, dtype=complex)
    for q in range(n):
        u = sla.expm(-0.5j * theta * embed({q: X})) @ u
    for a, b in graph.edges:
        u = sla.expm(0.25j * np.pi * embed({a: Z, b: Z})) @ u
    return u


@pytest.mark.parametrize("theta", [0.3, 0.9])
def test_statevector_matches_dense_unitary(theta):
    g = G.Graph(5, [(0, 1), (1, 2), (2, 3), (1, 4)], [0, 1, 0, 2])
    u = _dense_unitary(g, theta)
    psi0 = np.zeros(2 ** 5, dtype=complex)
    psi0[0] = 1
    want = np.linalg.matrix_power(u, 3) @ psi0
    got = S.evolve(g, theta, 3)
    assert np.allclose(got, want, atol=1e-12)


def test_statevector_clifford_string_is_phase():
    """<psi(pi/2, n')| S |psi(pi/2, n')> = sign for S = U^n' Z_i U^n'^dagger:
    ties the statevector's gate signs to the Clifford module (pinned above)."""
    _, g = G.hexagon_patches()
    for site, nprime in [(4, 2), (9, 3)]:
        s = C.string_from_z(g, site, nprime)
        psi = S.evolve(g, np.pi / 2, nprime)
        val = S.pauli_expectation(psi, g.n, s.ops)
        assert abs(val - s.phase) < 1e-12


def test_lightcone_matches_full_statevector():
    _, g = G.hexagon_patches()
    psi = S.evolve(g, 0.7, 3)
    ze = S.z_expectations(psi, g.n)
    for v in range(g.n):
        assert abs(S.lightcone_expectation(g, 0.7, 3, {v: "Z"}).real - ze[v]) < 1e-12


# ------------------------------------------------------------- BP oracle
def _paulis_vs_statevector(graph, chi, theta, steps):
    st = B.run(graph, chi, theta, steps)
    psi = S.evolve(graph, theta, steps)
    err = 0.0
    for v in range(graph.n):
        for lab in "XYZ":
            want = S.pauli_expectation(psi, graph.n, {v: lab}).real
            got = st.expect_1q(v, C.PAULI[lab]).real
            err = max(err, abs(got - want))
    return err, st


@pytest.mark.parametrize("graph", [G.path(8), G.star3_tree(),
                                   G.spanning_tree(G.hexagon_patches()[1])],
                         ids=["path8", "star7", "tree21"])
@pytest.mark.parametrize("theta", [0.3, np.pi / 4, 0.8])
def test_bp_exact_on_trees(graph, theta):
    """BP is exact on trees ("Model and Ansatz") when nothing is truncated."""
    steps = 4
    err, _ = _paulis_vs_statevector(graph, 2 ** steps, theta, steps)
    assert err < 1e-10


@pytest.mark.parametrize("steps", [3, 5])
@pytest.mark.parametrize("theta", [0.3, 0.8])
def test_bp_exact_short_circuits_on_a_loop(steps, theta):
    """For n < 6 steps BP agrees with exact dynamics (Results, first paragraph)."""
    err, _ = _paulis_vs_statevector(G.ring(12), 2 ** steps, theta, steps)
    assert err < 1e-10


def test_bp_exact_127_vs_lightcone():
    """127 qubits, no truncation, n = 4: equals the exact light-cone value."""
    g = G.eagle127()
    st = B.run(g, 16, 0.6, 4)
    for v in (0, 13, 30, 62, 100, 113, 126):
        want = S.lightcone_expectation(g, 0.6, 4, {v: "Z"}).real
        assert abs(st.expect_z(v) - want) < 1e-10


@pytest.mark.slow
def test_bp_exact_127_five_steps():
    """127 qubits after 5 steps, chi = 32 = 2^5: the paper's ~1e-14 regime."""
    g = G.eagle127()
    st = B.run(g, 32, 0.5, 5)
    for v in (13, 62, 113):
        want = S.lightcone_expectation(g, 0.5, 5, {v: "Z"}).real
        assert abs(st.expect_z(v) - want) < 1e-10


@pytest.mark.parametrize("steps", [1, 3, 6])
def test_theta_zero_closed_form(steps):
    st = B.run(G.eagle127(), 4, 0.0, steps)
    assert np.abs(st.all_z() - 1.0).max() < 1e-14


@pytest.mark.parametrize("steps", [1, 2, 4])
def test_theta_clifford_closed_form(steps):
    st = B.run(G.ring(12), 2 ** steps, np.pi / 2, steps)
    assert np.abs(st.all_z()).max() < 1e-12


def test_truncated_ring_differs_but_stays_physical():
    """chi = 8 < 2^5 truncates: results are approximate, yet every message is
    Hermitian PSD with unit norm and |<Z>| <= 1."""
    st = B.run(G.ring(12), 8, 0.8, 5)
    psi = S.evolve(G.ring(12), 0.8, 5)
    err = np.abs(st.all_z() - S.z_expectations(psi, 12)).max()
    assert 1e-6 < err < 1e-1
    for m in st.M.values():
        assert np.allclose(m, m.conj().T, atol=1e-14)
        assert abs(np.linalg.norm(m) - 1) < 1e-12
        assert np.linalg.eigvalsh(m).min() > -1e-12
    for v in range(12):
        r = st.rho(v)
        assert np.allclose(r, r.conj().T, atol=1e-12)
        assert abs(st.expect_z(v)) <= 1 + 1e-12


def test_gauge_invariance():
    """Inserting G G^-1 on a bond leaves every BP expectation unchanged."""
    st = B.run(G.ring(12), 8, 0.7, 4)
    ref = st.all_z()
    r = rng(5)
    e = 3
    v, w = st.g.edges[e]
    d = st.dim(e)
    gm = r.standard_normal((d, d)) + 1j * r.standard_normal((d, d)) + 3 * np.eye(d)
    gi = np.linalg.inv(gm)
    av, aw = st.leg_pos(v, e), st.leg_pos(w, e)
    st.T[v] = np.moveaxis(np.tensordot(st.T[v], gm, axes=(av, 0)), -1, av)
    st.T[w] = np.moveaxis(np.tensordot(st.T[w], gi.T, axes=(aw, 0)), -1, aw)
    st.bp_converge(1e-12, 2000)
    assert np.abs(st.all_z() - ref).max() < 1e-9


def test_bp_fixed_point_equation():
    """After convergence each message satisfies Eq. MessageTensorSelfConsistency
    written out with einsum (independent of the oracle's tensordot chain)."""
    st = B.run(G.star3_tree(), 8, 0.9, 3)
    st.bp_converge(1e-13, 500)
    v = 0
    e0, e1, e2 = st.g.legs[v]
    t = st.T[v]
    m1, m2 = st.incoming(v, e1), st.incoming(v, e2)
    out = np.einsum("pabc,pdef,be,cf->ad", t, t.conj(), m1, m2)
    out = 0.5 * (out + out.conj().T)
    out /= np.linalg.norm(out)
    assert np.allclose(out, st.M[(v, e0)], atol=1e-10)


def test_sqrt_pair_is_square_root():
    m = random_psd(rng(3), 6, rank=4)
    b, binv = B.BPState._sqrt_pair(m)
    assert np.allclose(b @ b, m, atol=1e-12)
    p = b @ binv
    assert np.allclose(p @ p, p, atol=1e-10)          # projector onto range(M)
    assert abs(np.trace(p).real - 4) < 1e-9


@pytest.mark.parametrize("site,nprime,steps", [(4, 2, 2), (9, 2, 3)])
def test_strings_region_and_extended_match_statevector(site, nprime, steps):
    """Both Pauli-string methods equal the exact value when nothing is truncated."""
    _, g = G.hexagon_patches()
    s = C.string_from_z(g, site, nprime)
    psi = S.evolve(g, 0.7, steps)
    want = S.pauli_expectation(psi, g.n, s.ops).real
    st = B.run(g, 2 ** (steps + nprime), 0.7, steps)
    reg = st.region_expectation(s.ops).real
    ext, _ = B.extended_string_expectation(st, site, nprime)
    assert abs(reg - want) < 1e-10
    assert abs(ext - want) < 1e-10


def test_periodic_cell_cover_invariance():
    """BP on the 5-site periodic cell equals BP on its 10-site double cover
    (a periodic cell is a unit cell of the infinite lattice, "Dynamics of the
    infinite heavy-hex lattice")."""
    base = G.periodic_cell()
    # double cover: copies i = 0, 1; the B - m3 edge crosses between copies
    edges, cols = [], []
    for i in range(2):
        off = 5 * i
        for (u, w), c in zip(base.edges, base.colours):
            if (u, w) == (1, 4):
                edges.append((1 + off, 4 + 5 * (1 - i)))
            else:
                edges.append((u + off, w + off))
            cols.append(c)
    cover = G.Graph(10, edges, cols)
    a = B.run(base, 4, 0.7, 3)
    b = B.run(cover, 4, 0.7, 3)
    za, zb = a.all_z(), b.all_z()
    assert np.allclose(zb[:5], za, atol=1e-10)
    assert np.allclose(zb[5:], za, atol=1e-10)


# ------------------------------------------------------------ Vidal gauge
from oracle import vidal as V  # noqa: E402


def _tree_side(g, e):
    u, w = g.edges[e]
    seen, stack = {u}, [u]
    while stack:
        v = stack.pop()
        for f in g.legs[v]:
            if f != e and g.other(f, v) not in seen:
                seen.add(g.other(f, v))
                stack.append(g.other(f, v))
    return sorted(seen)


def _schmidt(psi, n, side):
    t = psi.reshape([2] * n)  # axis n-1-q holds qubit q
    a = [n - 1 - q for q in side]
    b = [ax for ax in range(n) if ax not in a]
    return np.linalg.svd(np.transpose(t, a + b).reshape(2 ** len(side), -1), compute_uv=False)


def _contract_state(g, tensors, bond=None):
    """Full contraction of a small network into amplitudes psi[q_{n-1} .. q_0]
    (the statevector's ordering); bond[e] (optional) is a diagonal inserted on
    edge e."""
    letters = iter("abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ")
    phys = [next(letters) for _ in range(g.n)]
    elab = [next(letters) for _ in range(len(g.edges))]
    terms, ops = [], []
    for v in range(g.n):
        terms.append(phys[v] + "".join(elab[e] for e in g.legs[v]))
        ops.append(tensors[v])
    if bond is not None:
        for e in range(len(g.edges)):
            terms.append(elab[e])
            ops.append(bond[e])
    out = "".join(phys[q] for q in reversed(range(g.n)))
    return np.einsum(",".join(terms) + "->" + out, *ops, optimize=True).reshape(-1)


def test_vidal_canonical_on_tree_and_loopy_fixed_point():
    """Methods, "The Vidal gauge": contracting Gamma_v with lambda_x^2 on all
    legs but one and conj(Gamma_v) gives the identity on that leg; at a BP
    fixed point this holds on loopy graphs too (in the BP sense)."""
    for g, chi, steps in [(G.star3_tree(), 16, 3), (G.ring(12), 8, 5)]:
        st = B.run(g, chi, 0.6, steps)
        gam, lam = V.vidal_gauge(st)
        worst = 0.0
        for v in range(g.n):
            ll = [lam[e] for e in g.legs[v]]
            for j in range(len(ll)):
                worst = max(worst, V.canonical_residual(gam[v], ll, j))
        assert worst < 1e-8, (g.n, worst)


def test_vidal_lambda_are_schmidt_values_on_a_tree():
    """On a tree the Vidal bond weights are the state's Schmidt values across
    the edge (brute force: SVD of the statevector across the cut)."""
    g = G.star3_tree()
    st = B.run(g, 16, 0.7, 3)
    psi = S.evolve(g, 0.7, 3)
    _, lam = V.vidal_gauge(st)
    for e in range(len(g.edges)):
        sv = _schmidt(psi, g.n, _tree_side(g, e))
        sv = sv / np.linalg.norm(sv)
        k = len(lam[e])
        assert np.abs(lam[e] - sv[:k]).max() < 1e-10
        assert np.abs(sv[k:]).max(initial=0.0) < 1e-10


def test_vidal_form_reproduces_the_state():
    """Gamma and lambda (one lambda per edge between the Gammas) contract to the
    same state as the original tensors, up to one global factor."""
    g = G.star3_tree()
    st = B.run(g, 16, 0.9, 3)
    gam, lam = V.vidal_gauge(st)
    a = _contract_state(g, st.T)
    b = _contract_state(g, gam, bond=lam)
    c = np.vdot(b, a) / np.vdot(b, b)
    assert np.abs(a - c * b).max() < 1e-10 * np.abs(a).max()


def test_vidal_edge_gauge_undoes_to_identity():
    """A B^T = 1 on the support and both messages become diag(lambda)."""
    r = rng(7)
    d = 6
    x = r.standard_normal((d, d)) + 1j * r.standard_normal((d, d))
    y = r.standard_normal((d, d)) + 1j * r.standard_normal((d, d))
    m_uw, m_wu = x @ x.conj().T, y @ y.conj().T
    g_u, g_w, s = V.edge_gauge(m_uw, m_wu)
    a = g_u * np.sqrt(s)
    b = g_w * np.sqrt(s)
    assert np.abs(a @ b.T - np.eye(d)).max() < 1e-9
    assert np.abs(a.T @ m_uw @ a.conj() - np.diag(s)).max() < 1e-9 * s[0]
    assert np.abs(b.T @ m_wu @ b.conj() - np.diag(s)).max() < 1e-9 * s[0]


# ------------------------------------------------------- BP error estimate
from oracle import bperror as BE  # noqa: E402


def test_bp_error_vanishes_on_a_tree():
    """On a tree the cut norm network factorises: E = M_{u->w} (x) M_{w->u},
    rank one, so the estimate is zero."""
    g = G.star3_tree()
    st = B.run(g, 8, 0.7, 3)
    for e in range(len(g.edges)):
        err, s = BE.bp_error(st, e)
        assert err < 1e-12 and s[1] < 1e-10 * s[0]


def test_bp_error_of_a_uniform_ring_is_the_transfer_matrix_closed_form():
    """A ring of L equal site tensors, real and symmetric in their two legs:
    the transfer matrix T[(l l'), (r r')] = sum_p t[p,l,r] t[p,l',r'] is real
    symmetric, the symmetric gauge is an orthogonal change of the bond basis,
    and the cut ring is T^L, so the singular values of E are |mu_k|^L for the
    eigenvalues mu_k of T (the paper's exponential decay in the loop size)."""
    r = rng(5)
    chi = 3
    t = r.standard_normal((2, chi, chi))
    t = t + t.transpose(0, 2, 1)
    tm = np.einsum("plr,pms->lmrs", t, t).reshape(chi * chi, chi * chi)
    mu = np.linalg.eigvalsh(0.5 * (tm + tm.T))
    for L in (4, 6, 8):
        g = G.ring(L)
        st = B.BPState(g, chi)
        st.T = [t.astype(complex).copy() for _ in range(L)]
        st.M = {k: np.eye(chi, dtype=complex) / np.sqrt(chi) for k in st.M}
        st.bp_converge(tol=1e-13, max_iters=5000)
        err, s = BE.bp_error(st, 0)
        want = np.sort(np.abs(mu) ** L)[::-1]
        want = want / want[0]
        assert np.allclose(s / s[0], want, atol=1e-9)
        assert abs(err - (1 - np.sqrt(1 / np.sum(want ** 2)))) < 1e-9


def _cut_schmidt(psi, n, left):
    """Schmidt values and vectors of psi across the cut (left, rest); qubit q is
    bit q of the amplitude index."""
    right = [q for q in range(n) if q not in left]
    t = psi.reshape([2] * n)                      # axis i <-> qubit n-1-i
    axes = [n - 1 - q for q in left] + [n - 1 - q for q in right]
    m = np.transpose(t, axes).reshape(2 ** len(left), -1)
    u, s, vh = np.linalg.svd(m, full_matrices=False)
    return u, s, vh, axes


def _truncate_cut(psi, n, left, chi):
    """The best rank-chi approximation of psi across the cut, normalised."""
    u, s, vh, axes = _cut_schmidt(psi, n, left)
    m = (u[:, :chi] * s[:chi]) @ vh[:chi] / np.linalg.norm(s[:chi])
    t = m.reshape([2] * n)
    inv = np.argsort(axes)
    return np.transpose(t, inv).reshape(-1), s


@pytest.mark.parametrize("case", ["path8", "star7"])
def test_truncated_simple_update_is_the_optimal_schmidt_truncation(case):
    """Pin of the oracle's truncation branch (Methods, "The Vidal gauge" and "The
    simple update procedure").  On a tree the converged BP messages are the exact
    environments of each bond, so one simple update of exp(+i pi/4 Z_v Z_w) with a
    bond dimension below the edge's Schmidt rank must keep exactly the chi
    largest Schmidt values of the gated statevector across that edge, normalised,
    and the state it leaves must be the statevector's best rank-chi truncation
    across the cut: <Z_q> of every qubit agrees after BP regauges the tree."""
    if case == "path8":
        g = G.path(8)
        e, left = 3, [0, 1, 2, 3]                 # edge (3, 4)
    else:
        g = G.star3_tree()
        e, left = 0, [1, 2]                       # edge (0, 1): the arm {1, 2} against the rest
    theta, steps, chi_t = 0.7, 3, 3
    st = B.run(g, 64, theta, steps)              # exact: every bond below 2^steps <= 64
    psi = S.evolve(g, theta, steps)
    v, w = g.edges[e]
    s_v = 1 - 2 * ((np.arange(2 ** g.n) >> v) & 1)
    s_w = 1 - 2 * ((np.arange(2 ** g.n) >> w) & 1)
    psi_g = psi * np.exp(1j * np.pi / 4 * s_v * s_w)
    psi_t, s_full = _truncate_cut(psi_g, g.n, left, chi_t)
    assert np.count_nonzero(s_full > 1e-12 * s_full[0]) > chi_t       # the gate truncates
    assert (s_full[chi_t - 1] - s_full[chi_t]) / s_full[0] > 1e-3      # unique kept subspace
    st.chi = chi_t
    st.apply_zz(e, +1)
    kept = np.real(np.diag(st.M[(v, e)]))
    want = s_full[:chi_t] / np.linalg.norm(s_full[:chi_t])
    assert np.allclose(kept, want, atol=1e-10)
    assert abs(st.discarded[-1] - np.sum(s_full[chi_t:] ** 2) / np.sum(s_full ** 2)) < 1e-10
    st.bp_converge(1e-12, 1000)
    assert np.abs(st.all_z() - S.z_expectations(psi_t, g.n)).max() < 1e-10
