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


def test_shortest_policy_admits_small_jobs_first(tnlib):
    """One slot busy with a first job; then a large job and two small ones
    queue.  Under TN_SERVE_SHORTEST the small ones are admitted before the
    large one (oldest first would take the large one); results are those of
    the jobs alone."""
    g, p = OG.eagle127(), OG.falcon27_patch()
    with tnlib.Server(slots=1, policy="shortest") as srv:
        first = srv.submit(g.n, g.edges, g.colours, 16, 0.5, 3, prec="tf32")
        big = srv.submit(g.n, g.edges, g.colours, 32, 0.6, 4, prec="tf32")
        small = [srv.submit(p.n, p.edges, p.colours, 8, 0.3 + 0.1 * i, 2, prec="tf32")
                 for i in range(2)]
        srv.wait(first)
        zb, ib = srv.wait(big)
        outs = [srv.wait(t) for t in small]
    for (z, info), i in zip(outs, range(2)):
        assert info["queue_s"] < ib["queue_s"]
        assert np.abs(z - _alone(tnlib, p, 8, 0.3 + 0.1 * i, 2, "tf32")).max() <= 1e-12
    assert np.abs(zb - _alone(tnlib, g, 32, 0.6, 4, "tf32")).max() <= 1e-12


def test_unknown_policy_is_refused(tnlib):
    with pytest.raises(KeyError):
        tnlib.Server(slots=1, policy="random")


def test_job_over_budget_is_refused(tnlib):
    g = OG.eagle127()
    with tnlib.Server(slots=1, hbm_budget=1 << 20) as srv:
        with pytest.raises(tnlib.TNError) as ei:
            srv.submit(g.n, g.edges, g.colours, 16, 0.5, 1)
    assert ei.value.status == -2


def test_theta_chi_sweep_extrapolates_to_the_oracle(tnlib):
    """A theta grid x chi ladder as server jobs (FP32), extrapolated in 1/chi.
    At theta = 0 every <Z_v> is 1; at theta = 0.6 and 3 steps every chi >= 8 is
    exact for BP (bond dimension 2^3), so the slope vanishes and the intercept
    is the oracle's value (two points: A = 2 y(16) - y(8), so 3 x 1e-6)."""
    g = OG.falcon27_patch()
    thetas, chis = [0.0, 0.6], [8, 16]
    with tnlib.Server(slots=4) as srv:
        out = tnlib.theta_chi_sweep(srv, g.n, g.edges, g.colours, thetas, chis, 3, prec="fp32")
    assert (out["steps_done"] == 3).all()
    assert np.abs(out["z"][0] - 1.0).max() < 1e-6 and np.abs(out["z_inf"][0] - 1.0).max() < 3e-6
    want = OB.run(g, 8, 0.6, 3).all_z()
    assert np.abs(out["z_inf"][1] - want).max() < 3e-6
    assert np.abs(out["slope"][1]).max() < 1e-4
    # the intercepts are the straight line through the two chi points
    assert np.allclose(out["z_inf"], 2 * out["z"][:, 1] - out["z"][:, 0], atol=1e-12)


def test_served_job_returns_string_values(tnlib):
    """A job's Pauli strings (tn_job.ops) come back with its <Z_v>: the same
    values, by both methods, as tn_expect on a handle evolved alone (the
    paper's printed weight-10 string on 127 qubits and a weight-17 string)."""
    from oracle import clifford as OC
    n, edges, cols = tnlib.heavy_hex(7, 15)
    from oracle import graph as OG
    g = OG.eagle127()
    s10 = dict(OC.string_from_z(g, 13, 5).ops)
    s17 = dict(OC.string_from_z(g, 9, 5).ops)
    strings = [(s10, 1), (s17, -1)]   # both of the form U^n' Z_i U^-n' (method 1 needs that)
    chi, theta, steps = 8, 0.6, 5
    with tnlib.TNState(n, edges, cols, chi=chi) as s:
        s.apply_floquet(theta, steps)
        want = {m: s.expect(strings, method=m) for m in (0, 1)}
    with tnlib.Server(slots=2) as srv:
        t = {m: srv.submit(n, edges, cols, chi, theta, steps, ops=strings, method=m) for m in (0, 1)}
        for m in (0, 1):
            z, info = srv.wait(t[m])
            assert info["ops"].shape == (2,)
            assert np.abs(info["ops"] - want[m]).max() < 1e-12
