"""The Vidal-gauge export (tn_vidal_gauge, tn_get_gamma) against the FP64
oracle, the canonical conditions and, on a tree, the statevector.

Bounds: lambda_e comes from the FP32 messages through FP64 square roots and an
FP64 SVD, so it carries the messages' rounding, about 1e-6 of lambda_1 (2e-5
asserted).  Gamma divides by lambda on each leg, which amplifies that rounding
by lambda_1 / lambda_k: the canonical identity is asserted to 1e-3 on the
bond weights above 1e-3 lambda_1.  On a tree the state itself carries the
truncation solve's FP32-Gram floor (about 1e-4 sigma_1 on a zero Schmidt
value), so the comparison with the exact Schmidt values is held to 1e-4."""
import numpy as np
import pytest

from oracle import bptn as OB
from oracle import graph as OG
from oracle import statevector as OS
from oracle import vidal as OV

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tnlib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_14887_gb300 import build
    build.build()
    import paper_2306_14887_gb300 as tn
    return tn


def _side(g, e):
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
    t = psi.reshape([2] * n)
    a = [n - 1 - q for q in side]
    b = [ax for ax in range(n) if ax not in a]
    return np.linalg.svd(np.transpose(t, a + b).reshape(2 ** len(side), -1), compute_uv=False)


@pytest.mark.parametrize("name,chi,steps,theta", [("ring12", 8, 5, 0.6), ("patch27", 8, 4, 0.8)])
def test_lambda_matches_oracle(tnlib, name, chi, steps, theta):
    g = {"ring12": OG.ring(12), "patch27": OG.falcon27_patch()}[name]
    with tnlib.TNState(g.n, g.edges, g.colours, chi=chi) as s:
        s.apply_floquet(theta, steps)
        lam = s.vidal_gauge()
    o = OB.run(g, chi, theta, steps)
    assert o.min_gap > 1e-6
    _, want = OV.vidal_gauge(o)
    for e in range(len(g.edges)):
        w = np.zeros(chi)
        w[:len(want[e])] = want[e]
        assert np.abs(lam[e] - w).max() < 2e-5, (e, lam[e], w)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-3), ("tf32", 5e-2)])
def test_gamma_is_canonical(tnlib, prec, tol):
    """Sum of Gamma conj(Gamma) weighted by lambda^2 on the other legs is the
    identity (up to a factor) on each leg: eagle127 at chi = 16, 4 steps (a
    loopy graph at its BP fixed point).  In TF32 the messages are a fixed point
    only to the TF32 residual floor (BP stops near 2e-3), hence the wider
    bound there."""
    g = OG.eagle127()
    with tnlib.TNState(g.n, g.edges, g.colours, chi=16, prec=prec) as s:
        s.apply_floquet(0.6, 4)
        lam = s.vidal_gauge()
        worst = 0.0
        for v in list(range(0, 127, 9)) + [13, 62, 113]:
            gam = s.get_gamma(v).astype(np.complex128)
            legs = [lam[e] for e in g.legs[v]]
            for j in range(len(legs)):
                ll = list(legs)
                ll[j] = np.where(legs[j] > 1e-3 * legs[j][0], legs[j], 0.0)
                worst = max(worst, OV.canonical_residual(gam, ll, j))
    assert worst < tol, worst


def test_tree_lambda_are_schmidt_values_and_gamma_rebuilds_the_state(tnlib):
    g = OG.star3_tree()
    chi, steps, theta = 8, 3, 0.7
    with tnlib.TNState(g.n, g.edges, g.colours, chi=chi) as s:
        s.apply_floquet(theta, steps)
        lam = s.vidal_gauge()
        gam = [s.get_gamma(v).astype(np.complex128) for v in range(g.n)]
    psi = OS.evolve(g, theta, steps)
    for e in range(len(g.edges)):
        sv = _schmidt(psi, g.n, _side(g, e))
        sv = sv / np.linalg.norm(sv)
        k = min(chi, len(sv))
        assert np.abs(lam[e][:k] - sv[:k]).max() < 1e-4, (e, lam[e], sv)
    # Gamma with lambda on every edge contracts to the evolved state (up to a phase)
    letters = iter("abcdefghijklmnopqrstuvwxyz")
    phys = [next(letters) for _ in range(g.n)]
    elab = [next(letters) for _ in range(len(g.edges))]
    terms = [phys[v] + "".join(elab[e] for e in g.legs[v]) for v in range(g.n)]
    terms += [elab[e] for e in range(len(g.edges))]
    out = "".join(phys[q] for q in reversed(range(g.n)))
    amp = np.einsum(",".join(terms) + "->" + out, *gam, *[lam[e] for e in range(len(g.edges))],
                    optimize=True).reshape(-1)
    c = np.vdot(amp, psi) / np.vdot(amp, amp)
    assert np.abs(psi - c * amp).max() < 1e-4


def test_gamma_before_the_gauge_is_refused(tnlib):
    g = OG.star3_tree()
    with tnlib.TNState(g.n, g.edges, g.colours, chi=4) as s:
        with pytest.raises(tnlib.TNError):
            s.get_gamma(0)
