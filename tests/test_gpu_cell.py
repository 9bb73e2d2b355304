"""The periodic 5-site cell of the infinite heavy-hex lattice ("Dynamics of the
infinite heavy-hex lattice"): BP on the periodic cell is BP on the infinite
lattice, so the cell and its 10-site double cover give the same <Z>; large chi
(128, 256, bonds saturated) with the split-precision BF16 contractions against
the plain FP32 path at the same chi, and against the FP64 oracle where both run
(chi = 16, 64).
"""
import numpy as np
import pytest

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


def double_cover(base):
    edges, cols = [], []
    for i in range(2):
        off = 5 * i
        for (u, w), c in zip(base.edges, base.colours):
            if (u, w) == (1, 4):
                edges.append((1 + off, 4 + 5 * (1 - i)))
            else:
                edges.append((u + off, w + off))
            cols.append(c)
    return OG.Graph(10, edges, cols)


def _z(tn, g, chi, theta, steps, prec="fp32"):
    with tn.TNState(g.n, g.edges, g.colours, chi=chi, prec=prec) as s:
        s.apply_floquet(theta, steps)
        return s.expect_z_all()


def test_cell_equals_its_double_cover(tnlib):
    base = OG.periodic_cell()
    za = _z(tnlib, base, 16, 0.7, 8)
    zb = _z(tnlib, double_cover(base), 16, 0.7, 8)
    assert np.abs(zb[:5] - za).max() < 1e-6 and np.abs(zb[5:] - za).max() < 1e-6


@pytest.mark.parametrize("theta", [0.4, 1.0])
def test_cell_truncated_matches_oracle(tnlib, theta):
    g = OG.periodic_cell()
    o = OB.run(g, 16, theta, 7)
    z = _z(tnlib, g, 16, theta, 7)
    if o.min_gap > 1e-6:
        assert np.abs(z - o.all_z()).max() < 1e-6
    else:
        assert np.all(np.abs(z) <= 1 + 1e-6)


def test_cell_chi64_split_bf16_matches_oracle(tnlib):
    """Overlap point of the large-chi runs with the oracle: chi = 64."""
    g = OG.periodic_cell()
    o = OB.run(g, 64, 0.7, 7)
    z = _z(tnlib, g, 64, 0.7, 7, prec="bf16x3")
    assert np.abs(z - o.all_z()).max() < 1e-4


@pytest.mark.parametrize("chi,steps", [(128, 10), (256, 10)])
def test_cell_large_chi_split_bf16_matches_fp32_path(tnlib, chi, steps):
    """chi = 128 and 256 (site tensors 2 x chi^3, the 2chi x 2chi refined FP64
    truncation solve through its global-memory basis kernel) with every bond
    saturated: after 10 steps each of the cell's bonds keeps chi nonzero values.
    Split BF16 contractions against the plain FP32 path at the same chi."""
    g = OG.periodic_cell()
    out = {}
    for prec in ("bf16x3", "fp32"):
        with tnlib.TNState(g.n, g.edges, g.colours, chi=chi, prec=prec) as s:
            s.apply_floquet(0.7, steps)
            out[prec] = s.expect_z_all()
            if prec == "fp32":
                for e in range(len(g.edges)):
                    assert np.count_nonzero(s.bond_spectrum(e) > 1e-12) == chi
    assert np.abs(out["bf16x3"] - out["fp32"]).max() < 1e-4
    assert np.all(np.abs(out["fp32"]) <= 1 + 1e-6)
