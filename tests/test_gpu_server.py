"""Serving: continuous batching of jobs on one device (tn_server_*).

Jobs of different sizes, bond dimensions and precisions are submitted at once;
up to `slots` run concurrently, each on its own stream, admitted by HBM
footprint.  A job's result must be the same alone and in the mix: the library
shares no buffers between jobs and its kernels reduce in fixed orders, so the
stated tolerance here is 1e-12 (bitwise equality in practice).
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


JOBS = [  # graph, chi, theta, steps, prec
    (OG.falcon27_patch(), 8, 0.3, 4, "fp32"),
    (OG.ring(12), 8, 0.8, 5, "fp32"),
    (OG.heavy_hex(5, 11), 16, 0.6, 3, "tf32"),
    (OG.eagle127(), 8, 0.5, 4, "tf32"),
    (OG.falcon27_patch(), 16, 1.0, 3, "fp32"),
    (OG.eagle127(), 32, 0.7, 3, "tf32"),
    (OG.heavy_hex(5, 11), 8, 0.2, 5, "bf16"),
]


def _alone(tn, g, chi, theta, steps, prec):
    with tn.TNState(g.n, g.edges, g.colours, chi=chi, prec=prec) as s:
        s.apply_floquet(theta, steps)
        return s.expect_z_all()


def test_results_same_alone_and_in_the_mix(tnlib):
    with tnlib.Server(slots=3) as srv:
        tickets = [srv.submit(g.n, g.edges, g.colours, chi, th, st, prec=p)
                   for (g, chi, th, st, p) in JOBS]
        out = [srv.wait(t) for t in tickets]
        stats = srv.stats()
    assert stats["completed"] == len(JOBS) and stats["failed"] == 0
    assert stats["peak_resident"] >= 2          # jobs did run concurrently
    assert stats["peak_bytes"] <= stats["budget_bytes"]
    for (g, chi, th, st, p), (z, info) in zip(JOBS, out):
        assert info["steps_done"] == st and info["latency_s"] >= info["queue_s"] >= 0
        assert np.abs(z - _alone(tnlib, g, chi, th, st, p)).max() <= 1e-12


def test_sampled_job_matches_oracle(tnlib):
    g, chi, th, st = OG.falcon27_patch(), 8, 0.4, 3
    with tnlib.Server(slots=2) as srv:
        z, _ = srv.wait(srv.submit(g.n, g.edges, g.colours, chi, th, st))
    assert np.abs(z - OB.run(g, chi, th, st).all_z()).max() < 1e-6


def test_admission_by_footprint(tnlib):
    g = OG.eagle127()
    fp = tnlib.footprint_estimate(g.n, g.edges, g.colours, 16, "tf32")
    with tnlib.Server(slots=4, hbm_budget=int(1.5 * fp)) as srv:
        ts = [srv.submit(g.n, g.edges, g.colours, 16, 0.5 + 0.1 * i, 2, prec="tf32")
              for i in range(3)]
        res = [srv.wait(t) for t in ts]
        stats = srv.stats()
    assert all(r[1]["status"] == 0 for r in res)
    assert stats["peak_resident"] == 1          # only one fits the budget at a time
    assert stats["peak_bytes"] <= int(1.5 * fp)


def test_job_over_budget_is_refused(tnlib):
    g = OG.eagle127()
    with tnlib.Server(slots=1, hbm_budget=1 << 20) as srv:
        with pytest.raises(tnlib.TNError) as ei:
            srv.submit(g.n, g.edges, g.colours, 16, 0.5, 1)
    assert ei.value.status == -2
