"""The split-K autotuner (tn_autotune, tn_autotune_apply).

Tuning times the BP-sweep launches on the handle's own buffers; the sweep's
launches read the state and write only scratch, so the state is unchanged by
tuning, and the tuned handle evolves to the same result up to the order of the
FP32 partial sums.  A table written by one handle applies to another of the
same graph shape, chi and precision.
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


def _rows(table):
    return [ln.split() for ln in table.strip().splitlines() if ln.strip()]


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_tuning_leaves_the_state_and_keys_the_launches(tnlib, prec):
    g = OG.eagle127()
    with tnlib.TNState(g.n, g.edges, g.colours, chi=16, prec=prec) as s:
        s.apply_floquet(0.8, 5)
        before = [s.get_message(e, g.edges[e][0]).copy() for e in (0, 40, 100)]
        table = s.autotune(reps=3)
        after = [s.get_message(e, g.edges[e][0]) for e in (0, 40, 100)]
        for a, b in zip(before, after):
            assert np.array_equal(a, b)
        rows = _rows(table)
        assert rows, "no tunable launch"
        for r in rows:
            assert r[0] in ("close", "tile", "simt")
            assert int(r[7]) in (1, 2, 4, 8, 16, 32, 64) and float(r[8]) > 0
            if prec == "fp32":
                assert r[0] == "simt"


def test_tuned_evolution_matches_the_oracle(tnlib):
    """FP32, 127 qubits, chi = 16, truncated from step 5: the tuned handle
    stays within the FP32 bound of the oracle."""
    g = OG.eagle127()
    o = OB.run(g, 16, 1.0, 5)
    with tnlib.TNState(g.n, g.edges, g.colours, chi=16, prec="fp32") as s:
        s.apply_floquet(1.0, 2)
        s.autotune(reps=3)
        s.apply_floquet(1.0, 3)
        z = s.expect_z_all()
    if o.min_gap > 1e-6:
        assert np.abs(z - o.all_z()).max() < 1e-6


def test_table_applies_to_another_handle(tnlib, tmp_path):
    g = OG.eagle127()
    path = tmp_path / "tune.txt"
    with tnlib.TNState(g.n, g.edges, g.colours, chi=32, prec="tf32") as a:
        a.apply_floquet(0.7, 2)
        table = a.save_tuning(str(path), reps=3)
    rows = _rows(table)
    with tnlib.TNState(g.n, g.edges, g.colours, chi=32, prec="tf32") as b:
        assert b.load_tuning(str(path)) == len(rows)
        b.apply_floquet(0.7, 2)
        zb = b.expect_z_all()
    with tnlib.TNState(g.n, g.edges, g.colours, chi=32, prec="tf32") as c:
        c.apply_floquet(0.7, 2)
        # exact regime (chi >= 2^steps): TF32 rounding alone separates the runs
        assert np.abs(c.expect_z_all() - zb).max() < 1e-3
    # another chi: no key matches
    with tnlib.TNState(g.n, g.edges, g.colours, chi=16, prec="tf32") as d:
        assert d.apply_tuning(table) == 0


def test_batch_autotune_keeps_results(tnlib):
    """A union handle tuned on its initial state evolves to the untuned result
    up to the order of the FP32 partial sums."""
    gs = [OG.falcon27_patch(), OG.eagle127(), OG.heavy_hex(5, 11)]
    insts = [(g.n, g.edges, g.colours, 8, th) for g, th in zip(gs, (0.4, 0.9, 1.2))]
    out = []
    for tune in (False, True):
        with tnlib.Batch(insts, prec="fp32") as b:
            if tune:
                tables = b.autotune(reps=2)
                assert set(tables) == {8}
            b.evolve(4)
            out.append(b.expect_z())
    for za, zb in zip(*out):
        assert np.abs(za - zb).max() < 2e-6
