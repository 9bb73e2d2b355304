"""BP error estimate (tn_bp_error, Eq. BPErrorEstimate) against the FP64 oracle.

The library gauges on the device (FP32 state, FP64 gauge) and contracts the
cut norm network on the device in FP64; the oracle does both in FP64 from its
own evolution of the same circuit.  The two states agree to FP32 rounding, so
the normalised edge-environment spectra are compared to 1e-5 absolute."""
import numpy as np
import pytest

from oracle import bperror as OE
from oracle import bptn as OB
from oracle import graph as OG

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


def test_tree_edges_have_zero_bp_error(tnlib):
    g = OG.star3_tree()
    with tnlib.TNState(g.n, g.edges, g.colours, chi=8) as s:
        s.apply_floquet(0.7, 3)
        for e in range(len(g.edges)):
            err, sv = s.bp_error(e)
            assert err < 1e-6 and sv[1] < 1e-4 * sv[0]


def three_hexagons():
    """Three heavy hexagons in a row (30 qubits) cut from the 127-qubit layout."""
    one = [0, 1, 2, 3, 4, 14, 15, 18, 19, 20, 21, 22]
    two = one + [5, 6, 7, 8, 16, 23, 24, 25, 26]
    return OG.induced(OG.eagle127(), two + [9, 10, 11, 12, 17, 27, 28, 29, 30])


# truncated evolutions with visible loop correlations: BP errors of about
# 0.05 (12-ring), 0.19 (6-ring) and 1e-5 (two-hexagon patch)
@pytest.mark.parametrize("name,chi,steps,theta,edges", [
    ("ring12", 4, 6, 1.0, [0, 5]), ("ring6", 8, 5, 0.9, [0, 3]),
    ("patch27", 4, 5, 1.0, [0, 7, 20]), ("hex3", 4, 5, 1.0, [0, 11, 24, 31])])
def test_bp_error_matches_oracle(tnlib, name, chi, steps, theta, edges):
    g = {"ring12": OG.ring(12), "ring6": OG.ring(6), "patch27": OG.falcon27_patch(),
         "hex3": three_hexagons()}[name]
    with tnlib.TNState(g.n, g.edges, g.colours, chi=chi) as s:
        s.apply_floquet(theta, steps)
        got = {e: s.bp_error(e) for e in edges}
    o = OB.run(g, chi, theta, steps)
    assert o.min_gap > 1e-6
    for e in edges:
        err_w, sv_w = OE.bp_error(o, e)
        err, sv = got[e]
        k = min(len(sv), len(sv_w))
        assert abs(err - err_w) < 1e-5, (e, err, err_w)
        assert np.abs(sv[:k] / sv[0] - sv_w[:k] / sv_w[0]).max() < 1e-5


def test_large_network_is_refused(tnlib):
    g = OG.eagle127()
    with tnlib.TNState(g.n, g.edges, g.colours, chi=16) as s:
        s.apply_floquet(0.6, 4)
        with pytest.raises(tnlib.TNError):
            s.bp_error(0)
