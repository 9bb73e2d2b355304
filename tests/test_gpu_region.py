"""Weight-k Pauli strings by the BP-region method (tn_expect method 0) against
the FP64 oracle's region contraction on the same tree, and against the exact
statevector where BP is exact (a tree graph without truncation)."""
import numpy as np
import pytest

from oracle import bptn as OB
from oracle import clifford as OC
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


def _strings(g, weights, seed):
    r = np.random.default_rng(seed)
    out = []
    for w in weights:
        # connected-ish supports: a random site and its nearest sites by BFS order
        start = int(r.integers(g.n))
        seen, queue = [start], [start]
        while queue and len(seen) < 3 * w:
            v = queue.pop(0)
            for e in g.legs[v]:
                u = g.other(e, v)
                if u not in seen:
                    seen.append(u)
                    queue.append(u)
        sites = sorted(r.choice(seen, size=w, replace=False).tolist())
        out.append({int(q): "XYZ"[int(r.integers(3))] for q in sites})
    return out


@pytest.mark.parametrize("name,graph,chi,steps,theta", [
    ("ring12", OG.ring(12), 8, 4, 0.8),
    ("patch27", OG.falcon27_patch(), 8, 3, 0.6),
    ("eagle127", OG.eagle127(), 8, 4, 0.5),
])
def test_region_strings_match_oracle(tnlib, name, graph, chi, steps, theta):
    o = OB.run(graph, chi, theta, steps)
    strings = _strings(graph, [2, 3, 5, 8], seed=len(name))
    with tnlib.TNState(graph.n, graph.edges, graph.colours, chi=chi) as s:
        s.apply_floquet(theta, steps)
        got = s.expect([(ops, 1) for ops in strings], method=0)
    want = np.array([o.region_expectation(ops).real for ops in strings])
    assert np.abs(got - want).max() < 1e-6


def test_region_exact_on_a_tree(tnlib):
    """BP is exact on a tree without truncation: the region value is the exact
    expectation."""
    g = OG.star3_tree()
    chi, steps, theta = 8, 3, 0.7
    psi = OS.evolve(g, theta, steps)
    strings = [{0: "Z", 1: "X"}, {1: "Y", 2: "Z", 3: "X"}, {0: "X", 4: "Z", 6: "Y"}]
    with tnlib.TNState(g.n, g.edges, g.colours, chi=chi) as s:
        s.apply_floquet(theta, steps)
        got = s.expect([(ops, 1) for ops in strings], method=0)
    for ops, val in zip(strings, got):
        exact = OS.pauli_expectation(psi, g.n, ops)
        assert abs(val - exact) < 1e-6


def test_region_printed_weight10_string(tnlib):
    """The paper's weight-10 string on 127 qubits after 5 steps: the region
    value against the oracle's region value (same tree)."""
    g = OG.eagle127()
    s10 = OC.string_from_z(g, 13, 5)
    ops = dict(s10.ops)
    assert len(ops) == 10
    o = OB.run(g, 8, 0.4, 5)
    want = o.region_expectation(ops).real
    with tnlib.TNState(g.n, g.edges, g.colours, chi=8) as s:
        s.apply_floquet(0.4, 5)
        got = s.expect([(ops, 1)], method=0)[0]
    assert abs(got - want) < 1e-6


@pytest.mark.parametrize("prec,tol", [("tf32", 5e-3), ("tf32x3", 3e-5)])
def test_region_tensor_core_modes(tnlib, prec, tol):
    g = OG.falcon27_patch()
    o = OB.run(g, 16, 0.6, 4)
    strings = _strings(g, [2, 4, 6], seed=9)
    with tnlib.TNState(g.n, g.edges, g.colours, chi=16, prec=prec) as s:
        s.apply_floquet(0.6, 4)
        got = s.expect([(ops, 1) for ops in strings], method=0)
    want = np.array([o.region_expectation(ops).real for ops in strings])
    assert np.abs(got - want).max() < tol


def weight17_generator(g, nprime=5):
    """The first qubit i (in increasing order) whose string
    U^n'(pi/2) Z_i U^n'(pi/2)^dagger has weight 17, for the extended-evolution
    depth n' = 5 of the printed weight-10 string: the reading of the weight-17
    observable, whose support the paper does not print."""
    for i in range(g.n):
        s = OC.string_from_z(g, i, nprime)
        if len(s.ops) == 17:
            return i, s
    raise AssertionError("no weight-17 string")


def test_weight17_string_both_methods_match_oracle(tnlib):
    """A weight-17 string on 127 qubits after 5 steps (chi = 8, truncating from
    step 4), by the BP region (method 0) and by extended evolution (method 1),
    each against the oracle's same method ("Measuring expectation values")."""
    g = OG.eagle127()
    site, s17 = weight17_generator(g)
    ops = dict(s17.ops)
    assert (site, len(ops)) == (9, 17)
    chi, theta, steps = 8, 0.4, 5
    o = OB.run(g, chi, theta, steps)
    want_region = o.region_expectation(ops).real
    want_ext, _ = OB.extended_string_expectation(o, site, 5)
    with tnlib.TNState(g.n, g.edges, g.colours, chi=chi) as s:
        s.apply_floquet(theta, steps)
        got_region = s.expect([(ops, 1)], method=0)[0]
        got_ext = s.expect([(ops, 1)], method=1)[0]
    assert abs(got_region - want_region) < 1e-6
    assert abs(got_ext - want_ext) < 1e-6
