"""The Vidal gauge of a BP-gauged tensor-network state, in FP64 (test infrastructure).

Methods, "The Vidal gauge": a tree tensor network in the Vidal gauge is a
tensor Gamma_v per site and a diagonal, non-negative bond matrix lambda_e per
edge, such that contracting Gamma_v with lambda_x^2 on all legs but one, and
with conj(Gamma_v), gives the identity on the remaining leg; the BP messages
at their fixed point define the gauge transformation that brings the network
there (exactly on trees, and as the BP approximation on loopy graphs).

Written out for one edge e = (u, w), with M_{u->w} the message u sends across
e (indexed [ket, bra], as in `bptn`):
  P = M_{u->w}^1/2, Q = M_{w->u}^1/2         Hermitian square roots
  Q^T P = U diag(lambda) V^H                 SVD
  A = Q conj(U) lambda^-1/2 on u's leg, B = P V lambda^-1/2 on w's leg
satisfy A B^T = 1 on the messages' support and turn both messages into
diag(lambda).  Writing each gauged site tensor as Gamma_v with lambda^1/2 on
every leg gives Gamma_v = T_v contracted leg by leg with Q conj(U) / lambda
(u side) or P V / lambda (w side).  lambda is returned with unit 2-norm.
"""
from __future__ import annotations

import numpy as np

LAMBDA_CUT = 1e-12   # relative to lambda_1; below it a bond weight counts as zero
EIG_CUT = 1e-14      # relative to the largest message eigenvalue


def hermitian_sqrt(m):
    """Square root of a Hermitian PSD message (negative rounding dropped)."""
    m = 0.5 * (m + m.conj().T)
    lam, w = np.linalg.eigh(m)
    keep = lam > EIG_CUT * max(lam.max(), 0.0)
    r = np.where(keep, np.sqrt(np.where(keep, lam, 0.0)), 0.0)
    return (w * r) @ w.conj().T


def edge_gauge(m_uw, m_wu):
    """(G_u, G_w, lambda) for one edge from its two messages: the leg matrices
    applied to u's and w's leg (rows: the old bond index) and the unnormalised
    bond weights, decreasing."""
    p = hermitian_sqrt(m_uw)
    q = hermitian_sqrt(m_wu)
    u, s, vh = np.linalg.svd(q.T @ p)
    keep = s > LAMBDA_CUT * s[0] if s[0] > 0 else np.zeros_like(s, dtype=bool)
    inv = np.where(keep, 1.0 / np.where(keep, s, 1.0), 0.0)
    g_u = (q @ u.conj()) * inv
    g_w = (p @ vh.conj().T) * inv
    return g_u, g_w, np.where(keep, s, 0.0)


def vidal_gauge(state):
    """(Gamma list, lambda dict) of a `bptn.BPState` from its current messages.
    lambda[e] has unit 2-norm."""
    g = state.g
    gmat = {}
    lam = {}
    for e, (u, w) in enumerate(g.edges):
        g_u, g_w, s = edge_gauge(state.M[(u, e)], state.M[(w, e)])
        gmat[(u, e)] = g_u
        gmat[(w, e)] = g_w
        lam[e] = s / np.linalg.norm(s)
    gammas = []
    for v in range(g.n):
        x = state.T[v]
        for e in g.legs[v]:
            ax = state.leg_pos(v, e)
            x = np.moveaxis(np.tensordot(x, gmat[(v, e)], axes=(ax, 0)), -1, ax)
        gammas.append(x)
    return gammas, lam


def canonical_residual(gamma, legs_lambda, leg):
    """|| C / mean(diag C) - 1 || on the support of the leg's own lambda, with
    C[k, k'] = sum over the other indices of Gamma[..k..] conj(Gamma[..k'..])
    prod_{x != leg} lambda_x^2.  gamma: (2, d_1, .., d_m); legs_lambda: the
    lambda of each virtual leg in order; leg: 0-based virtual leg index."""
    x = gamma.copy()
    for j, lam in enumerate(legs_lambda):
        if j == leg:
            continue
        shape = [1] * x.ndim
        shape[1 + j] = -1
        x = x * lam.reshape(shape)
    ax = 1 + leg
    others = [i for i in range(x.ndim) if i != ax]
    c = np.tensordot(x, x.conj(), axes=(others, others))
    sup = legs_lambda[leg] > 0
    c = c[np.ix_(sup, sup)]
    c = c / np.mean(np.diag(c).real)
    return np.abs(c - np.eye(c.shape[0])).max()
