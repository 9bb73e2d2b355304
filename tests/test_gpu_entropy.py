"""Bond spectra and the entanglement entropy per edge (the infinite-lattice
paragraph's Eq. EntanglementEntropy, read s = -sum lambda^2 log2 lambda^2).

On a tree without truncation, BP-gauged simple update keeps the exact Schmidt
values across each edge: a gate on any other edge acts on one side of the cut
only, so the spectrum the solve kept at the edge's gate is the state's Schmidt
spectrum across that edge at the end of the step."""
import numpy as np
import pytest

from oracle import graph as OG
from oracle import statevector as OS

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


def side_of(g, e):
    u, w = g.edges[e]
    seen, stack = {u}, [u]
    while stack:
        v = stack.pop()
        for f in g.legs[v]:
            if f == e:
                continue
            x = g.other(f, v)
            if x not in seen:
                seen.add(x)
                stack.append(x)
    assert w not in seen
    return sorted(seen)


def schmidt(psi, n, side):
    t = psi.reshape([2] * n)  # axis n-1-q holds qubit q
    a = [n - 1 - q for q in side]
    b = [ax for ax in range(n) if ax not in a]
    m = np.transpose(t, a + b).reshape(2 ** len(side), -1)
    return np.linalg.svd(m, compute_uv=False)


# The solve works from FP32 Gram matrices G = X^H X: an eigenvalue of G is
# known to about eps_32 ||G||, so a singular value to about sqrt(eps_32)
# sigma_1 ~ 1e-4 sigma_1 absolute; a zero Schmidt value shows up at that
# level (its weight, ~1e-9, is below every other error of the state).
@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("tf32x3", 1e-4)])
def test_tree_bond_spectra_are_schmidt_values(tnlib, prec, tol):
    g = OG.star3_tree()
    chi, steps, theta = 8, 3, 0.7
    psi = OS.evolve(g, theta, steps)
    with tnlib.TNState(g.n, g.edges, g.colours, chi=chi, prec=prec) as s:
        s.apply_floquet(theta, steps)
        for e in range(len(g.edges)):
            got = s.bond_spectrum(e)
            want = np.zeros(chi)
            sv = schmidt(psi, g.n, side_of(g, e))[:chi]
            want[:len(sv)] = sv
            assert np.abs(got - want).max() < tol
            ent = s.entanglement_entropy(e)
            p = want ** 2
            assert abs(ent - float(-(p[p > 0] * np.log2(p[p > 0])).sum())) < 1e-5


def test_product_state_spectrum(tnlib):
    g = OG.periodic_cell()
    with tnlib.TNState(g.n, g.edges, g.colours, chi=8) as s:
        s.apply_floquet(0.0, 2)
        for e in range(len(g.edges)):
            sp = s.bond_spectrum(e)
            assert abs(sp[0] - 1.0) < 1e-7 and np.abs(sp[1:]).max() < 1e-7
            assert abs(s.entanglement_entropy(e)) < 1e-6


def test_cell_spectra_are_normalised_and_sorted(tnlib):
    g = OG.periodic_cell()
    with tnlib.TNState(g.n, g.edges, g.colours, chi=16) as s:
        s.apply_floquet(0.7, 6)
        for e in range(len(g.edges)):
            sp = s.bond_spectrum(e)
            assert abs((sp ** 2).sum() - 1.0) < 1e-6
            assert np.all(np.diff(sp) <= 1e-12) and sp.min() >= 0
            assert 0.0 < s.entanglement_entropy(e) <= np.log2(16) + 1e-9
