"""Checkpoint / resume: a job saved after some steps and restored (into the same
handle or a fresh one on the same graph) continues exactly as the uninterrupted
job: every kernel reduces in a fixed order, so resumed results are bitwise
equal."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("prec,chi", [("fp32", 8), ("tf32", 32)])
def test_resume_is_bitwise_identical(tnlib, prec, chi):
    g = OG.eagle127()
    with tnlib.TNState(g.n, g.edges, g.colours, chi=chi, prec=prec) as a:
        a.apply_floquet(0.7, 3)
        image = a.save_state()
        a.apply_floquet(0.7, 2)
        z_straight = a.expect_z_all()
        s_straight = a.bond_spectrum(5)
        # back to the saved point in the same handle
        a.load_state(image)
        a.apply_floquet(0.7, 2)
        assert np.array_equal(a.expect_z_all(), z_straight)
    # and in a fresh handle on the same graph
    with tnlib.TNState(g.n, g.edges, g.colours, chi=chi, prec=prec) as b:
        b.load_state(image)
        b.apply_floquet(0.7, 2)
        assert np.array_equal(b.expect_z_all(), z_straight)
        assert np.array_equal(b.bond_spectrum(5), s_straight)


def test_load_rejects_another_graph_or_chi(tnlib):
    g = OG.ring(12)
    with tnlib.TNState(g.n, g.edges, g.colours, chi=8) as a:
        a.apply_floquet(0.5, 1)
        image = a.save_state()
    with tnlib.TNState(g.n, g.edges, g.colours, chi=16) as b:
        with pytest.raises(tnlib.TNError) as ei:
            b.load_state(image)
        assert ei.value.status == -1
    h = OG.falcon27_patch()
    with tnlib.TNState(h.n, h.edges, h.colours, chi=8) as c:
        with pytest.raises(tnlib.TNError):
            c.load_state(image)
        with pytest.raises(tnlib.TNError):
            c.load_state(image[:40])
