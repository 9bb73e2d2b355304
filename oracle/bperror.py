"""BP error estimate of an edge, in FP64 (test infrastructure).

Methods, "Estimating the error of BP for general tensor networks" and Eq.
"BPErrorEstimate": bring the state to the symmetric gauge (the Vidal gauge
with lambda^1/2 on every leg), form the norm network (each site's tensor and
its conjugate, physical index summed), split the chosen edge's index into the
part on each endpoint and contract everything else: the edge environment E, a
chi^2 x chi^2 matrix.  BP treats E as rank one; with E's singular values s the
estimate is 1 - sqrt(s_1^2 / sum s_i^2) (one minus the square root of the
index of separability).  Exact contraction: small networks only.
"""
from __future__ import annotations

import numpy as np

from . import vidal


def symmetric_gauge(state):
    """Site tensors of the symmetric gauge (Gamma with lambda^1/2 on every leg),
    each bond cut to the support of its lambda, and the lambdas."""
    gam, lam = vidal.vidal_gauge(state)
    g = state.g
    sup = {e: int(np.count_nonzero(lam[e] > 0)) for e in lam}
    out = []
    for v in range(g.n):
        t = gam[v]
        for e in g.legs[v]:
            ax = state.leg_pos(v, e)
            t = np.take(t, np.arange(sup[e]), axis=ax)
            shape = [1] * t.ndim
            shape[ax] = -1
            t = t * np.sqrt(lam[e][:sup[e]]).reshape(shape)
        out.append(t)
    return out, lam


def edge_environment(state, e):
    """E[(u side), (w side)] of edge e = (u, w) in the symmetric gauge."""
    g = state.g
    ts, _ = symmetric_gauge(state)
    letters = iter("abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ")
    lab = {f: next(letters) for f in range(len(g.edges)) if f != e}
    cu, cw = next(letters), next(letters)
    u, w = g.edges[e]
    terms, ops = [], []
    for v in range(g.n):
        t = ts[v]
        d = t.ndim - 1
        # double layer D[(l_1 l_1'), ..] = sum_p t[p, l..] conj(t[p, l'..])
        dl = np.tensordot(t, t.conj(), axes=([0], [0]))           # l_1..l_d, l_1'..l_d'
        perm = [i for j in range(d) for i in (j, d + j)]
        dl = np.transpose(dl, perm).reshape([t.shape[1 + j] ** 2 for j in range(d)])
        s = ""
        for f in g.legs[v]:
            s += lab[f] if f != e else (cu if v == u else cw)
        terms.append(s)
        ops.append(dl)
    return np.einsum(",".join(terms) + "->" + cu + cw, *ops, optimize="greedy")


def bp_error(state, e):
    """(1 - sqrt(s_1^2 / sum s^2), s) for edge e (Eq. BPErrorEstimate)."""
    s = np.linalg.svd(edge_environment(state, e), compute_uv=False)
    return 1.0 - np.sqrt(s[0] ** 2 / np.sum(s ** 2)), s
