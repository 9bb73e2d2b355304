"""Batched instances: many independent heavy-hex instances of uneven size, each
with its own kick angle, evolved as one handle over their disjoint union.

BP and the simple update never couple components of a graph, so each instance
evolves as it would alone; the union only changes how the work is launched
(every contraction of every instance in the same launches, one CUDA graph per
BP sweep).  The BP stop rule acts on the largest residual over the union, so an
instance may receive sweeps beyond its own stopping point: at the FP32 floor
these move <Z> by well under the FP32 parity bound of 1e-6.
"""
import numpy as np
import pytest

from oracle import bptn as OB
from oracle import graph as OG
from workloads import batched_jobs

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


GRAPHS = {27: OG.falcon27_patch, 65: lambda: OG.heavy_hex(5, 11), 127: OG.eagle127,
          433: lambda: OG.heavy_hex(13, 27)}


def _instances(n_inst, seed=20230626):
    jobs = batched_jobs(n=n_inst, seed=seed)
    return [(GRAPHS[size](), theta) for (size, _chi, theta, _steps) in jobs]


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-6), ("tf32", 5e-3)])
def test_union_matches_each_instance_alone(tnlib, prec, tol):
    insts = _instances(8)
    chi, steps = 8, 3
    n, edges, cols, offs = tnlib.batch_union([(g.n, g.edges, g.colours) for g, _ in insts])
    thetas = np.concatenate([np.full(g.n, th) for g, th in insts])
    with tnlib.TNState(n, edges, cols, chi=chi, prec=prec) as s:
        s.apply_floquet_field(thetas, steps)
        z = s.expect_z_all()
        union_launches = s.stats()["kernel_launches"]
    alone_launches = 0
    for (g, th), off in zip(insts, offs):
        with tnlib.TNState(g.n, g.edges, g.colours, chi=chi, prec=prec) as a:
            a.apply_floquet(th, steps)
            za = a.expect_z_all()
            alone_launches += a.stats()["kernel_launches"]
        assert np.abs(z[off:off + g.n] - za).max() < tol
    # one set of launches for all instances instead of one per instance
    assert union_launches < alone_launches / 2


def test_union_instance_matches_oracle(tnlib):
    """Exact regime (chi >= 2^steps): every instance of the union against the
    FP64 oracle run on that instance alone."""
    insts = _instances(4, seed=3)
    chi, steps = 8, 3
    n, edges, cols, offs = tnlib.batch_union([(g.n, g.edges, g.colours) for g, _ in insts])
    thetas = np.concatenate([np.full(g.n, th) for g, th in insts])
    with tnlib.TNState(n, edges, cols, chi=chi) as s:
        s.apply_floquet_field(thetas, steps)
        z = s.expect_z_all()
    for (g, th), off in zip(insts, offs):
        if g.n > 127:
            continue
        want = OB.run(g, chi, th, steps).all_z()
        assert np.abs(z[off:off + g.n] - want).max() < 1e-6


def test_field_with_uniform_angle_equals_scalar_kick(tnlib):
    g = OG.ring(12)
    with tnlib.TNState(g.n, g.edges, g.colours, chi=8) as a, \
            tnlib.TNState(g.n, g.edges, g.colours, chi=8) as b:
        a.apply_floquet(0.7, 4)
        b.apply_floquet_field(np.full(g.n, 0.7), 4)
        assert np.abs(a.expect_z_all() - b.expect_z_all()).max() < 1e-6
