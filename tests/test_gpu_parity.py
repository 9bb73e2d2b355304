"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: the bound for the plain FP32 path is |d<Z>| <= 1e-6
against the FP64 oracle; single kernels (one BP sweep, rho) are compared
element by element at 2e-5 absolute on unit-norm messages, a few FP32 ulps
times the contraction length.
"""
import numpy as np
import pytest

from oracle import bptn as OB
from oracle import clifford as OC
from oracle import graph as OG
from oracle import statevector as OS
from test_gpu_headline import check_valid_state
from workloads import THETA_SMALL, random_state

pytestmark = pytest.mark.gpu

Z_TOL = 1e-6
# the shared-memory solve runs its Jacobi rotations in FP32 (stated bound)
Z_TOL_SHARED = 1e-5
MSG_TOL = 2e-5


@pytest.fixture(scope="module")
def tnlib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_14887_gb300 import build
    build.build()
    import paper_2306_14887_gb300 as tn
    return tn


def make(tn, g, chi, **kw):
    return tn.TNState(g.n, g.edges, g.colours, chi=chi, **kw)


def oracle_from_arrays(g, chi, tensors, msgs):
    st = OB.BPState(g, chi)
    st.T = [t.astype(complex) for t in tensors]
    st.M = {k: m.astype(complex) for k, m in msgs.items()}
    return st


GRAPHS = {
    "ring12": OG.ring(12),
    "star7": OG.star3_tree(),
    "path5": OG.path(5),
    "patch27": OG.falcon27_patch(),
}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("chi", [3, 8, 16])
def test_one_bp_sweep_matches_oracle(tnlib, name, chi):
    g = GRAPHS[name]
    tensors, msgs = random_state([g.degree(v) for v in range(g.n)], g.edges, chi, seed=11)
    s = make(tnlib, g, chi)
    for v in range(g.n):
        s.set_site(v, tensors[v])
    for (src, e), m in msgs.items():
        s.set_message(e, src, m)
    it, res, _ = s.bp_converge(tol=1e30, max_iters=1)
    assert it == 1
    o = oracle_from_arrays(g, chi, tensors, msgs)
    want_res = o.bp_sweep()
    assert abs(res - want_res) < 1e-4 * max(1.0, want_res)
    err = max(np.abs(s.get_message(e, src) - o.M[(src, e)]).max() for (src, e) in o.M)
    assert err < MSG_TOL
    s.close()


@pytest.mark.parametrize("name", ["star7", "patch27"])
def test_single_site_paulis_match_oracle(tnlib, name):
    g = GRAPHS[name]
    chi = 8
    tensors, msgs = random_state([g.degree(v) for v in range(g.n)], g.edges, chi, seed=5)
    s = make(tnlib, g, chi)
    for v in range(g.n):
        s.set_site(v, tensors[v])
    for (src, e), m in msgs.items():
        s.set_message(e, src, m)
    o = oracle_from_arrays(g, chi, tensors, msgs)
    strings = [({v: lab}, 1) for v in range(g.n) for lab in "XYZ"]
    got = s.expect(strings)
    want = np.array([o.expect_1q(v, OC.PAULI[lab]).real for v in range(g.n) for lab in "XYZ"])
    assert np.abs(got - want).max() < 1e-5
    s.close()


@pytest.mark.parametrize("theta", THETA_SMALL)
def test_ring12_floquet_matches_oracle(tnlib, theta):
    """12-qubit ring, chi = 8, 5 steps (truncation from step 4), BP tol 1e-10.

    Where the oracle logs a truncation with a relative gap sigma_chi - sigma_chi+1
    below 1e-6 (the flat spectra of the Clifford point theta = pi/2), the kept
    subspace is not unique and several results are correct: there only the
    properties every valid result has are checked."""
    g = OG.ring(12)
    o = OB.run(g, 8, theta, 5)
    s = make(tnlib, g, 8)
    s.apply_floquet(theta, 5)
    z = s.expect_z_all()
    if o.min_gap > 1e-6:
        assert np.abs(z - o.all_z()).max() < Z_TOL
    else:
        check_valid_state(s, g, 2e-6)
    if theta == 0.0:
        assert np.abs(z - 1.0).max() < Z_TOL
    s.close()


def test_clifford_point_without_truncation_is_exact(tnlib):
    """theta = pi/2 with chi = 2^steps: <Z_v> = 0 exactly (Clifford point)."""
    g = OG.ring(12)
    s = make(tnlib, g, 16)
    s.apply_floquet(np.pi / 2, 4)
    assert np.abs(s.expect_z_all()).max() < Z_TOL
    s.close()


@pytest.mark.parametrize("steps", [0, 1, 3, 5])
def test_ring12_exact_regime_matches_statevector(tnlib, steps):
    g = OG.ring(12)
    s = make(tnlib, g, 32)
    s.apply_floquet(0.8, steps)
    z = s.expect_z_all()
    exact = OS.z_expectations(OS.evolve(g, 0.8, steps), 12)
    assert np.abs(z - exact).max() < Z_TOL
    s.close()


def test_path_with_degree_one_ends(tnlib):
    g = OG.path(7)
    s = make(tnlib, g, 16)
    s.apply_floquet(0.7, 4)
    exact = OS.evolve(g, 0.7, 4)
    z = s.expect_z_all()
    assert np.abs(z - OS.z_expectations(exact, g.n)).max() < Z_TOL
    xy = s.expect([({v: l}, 1) for v in range(g.n) for l in "XY"])
    want = [OS.pauli_expectation(exact, g.n, {v: l}).real for v in range(g.n) for l in "XY"]
    assert np.abs(xy - np.array(want)).max() < Z_TOL
    s.close()


def test_eagle127_exact_regime_matches_lightcone(tnlib):
    """127 qubits, 4 steps at chi = 16 = 2^4: BP is exact (no loop reached)."""
    g = OG.eagle127()
    s = make(tnlib, g, 16)
    s.apply_floquet(0.6, 4)
    z = s.expect_z_all()
    o = OB.run(g, 16, 0.6, 4)
    assert np.abs(z - o.all_z()).max() < Z_TOL
    for v in (0, 13, 62, 113):
        assert abs(z[v] - OS.lightcone_expectation(g, 0.6, 4, {v: "Z"}).real) < Z_TOL
    s.close()


# theta_h of the bench's sweep point: the tenth of 16 points on [0, pi/2]
BENCH_THETA = float(np.linspace(0.0, np.pi / 2, 16)[9])


@pytest.mark.parametrize("chi", [32, 64])
def test_bench_configuration_exact_regime_fp32(tnlib, chi):
    """The bench workload (127 qubits, chi = 64) for its first 5 steps in FP32.

    Bonds reach at most 2^5 = 32, so nothing is truncated and BP is exact
    (the backward light cone of one site after 5 steps holds no loop of the
    12-site heavy-hex cells); chi = 64 also exercises the zero-padded bonds.
    All 127 <Z_v> against the FP64 oracle, a spread of sites against the
    light-cone statevector.
    """
    g = OG.eagle127()
    s = make(tnlib, g, chi)
    s.apply_floquet(BENCH_THETA, 5)
    z = s.expect_z_all()
    s.close()
    o = OB.run(g, 32, BENCH_THETA, 5)
    assert np.abs(z - o.all_z()).max() < Z_TOL
    for v in (0, 6, 13, 44, 62, 113, 126):
        assert abs(z[v] - OS.lightcone_expectation(g, BENCH_THETA, 5, {v: "Z"}).real) < Z_TOL


@pytest.mark.parametrize("solve,tol", [("fp64", Z_TOL), ("shared", Z_TOL_SHARED)])
def test_eagle127_truncated_matches_oracle(tnlib, solve, tol):
    """127 qubits, chi = 4 < 2^5: truncation in every gate from step 3."""
    g = OG.eagle127()
    o = OB.run(g, 4, 0.8, 5)
    assert o.min_gap > 1e-6      # no near-ties at the truncation boundary
    s = make(tnlib, g, 4, solve=solve)
    s.apply_floquet(0.8, 5)
    assert np.abs(s.expect_z_all() - o.all_z()).max() < tol
    s.close()


@pytest.mark.parametrize("theta", [0.3, 0.8])
@pytest.mark.parametrize("chi,steps", [(8, 5), (32, 5)])
def test_ring12_shared_solve_within_stated_bound(tnlib, theta, chi, steps):
    g = OG.ring(12)
    o = OB.run(g, chi, theta, steps)
    s = make(tnlib, g, chi, solve="shared")
    s.apply_floquet(theta, steps)
    assert np.abs(s.expect_z_all() - o.all_z()).max() < Z_TOL_SHARED
    s.close()


@pytest.mark.parametrize("chi,steps,theta", [(8, 6, 0.6), (16, 5, 1.0)])
def test_eagle127_deeper_truncated_matches_oracle(tnlib, chi, steps, theta):
    g = OG.eagle127()
    o = OB.run(g, chi, theta, steps)
    s = make(tnlib, g, chi)
    s.apply_floquet(theta, steps)
    z = s.expect_z_all()
    if o.min_gap > 1e-6:
        assert np.abs(z - o.all_z()).max() < Z_TOL
    else:
        # a near-tie at a truncation: several results are correct, so only what
        # every valid result has is checked
        check_valid_state(s, g, 2e-6)
    s.close()


def test_extended_evolution_string_matches_statevector(tnlib):
    _, g = OG.hexagon_patches()
    site, nprime, steps, theta = 9, 2, 2, 0.7
    sref = OC.string_from_z(g, site, nprime)
    want = OS.pauli_expectation(OS.evolve(g, theta, steps), g.n, sref.ops).real
    s = make(tnlib, g, 16)
    s.apply_floquet(theta, steps)
    got = s.expect([(sref.ops, 1)], method=1)[0]
    assert abs(got - want) < Z_TOL
    # the state is restored after the measurement
    z_before = s.expect_z_all()
    s.expect([(sref.ops, 1)], method=1)
    assert np.abs(s.expect_z_all() - z_before).max() < 1e-7
    s.close()


def test_messages_are_hermitian_unit_norm(tnlib):
    g = OG.ring(12)
    s = make(tnlib, g, 8)
    s.apply_floquet(0.8, 6)
    for e, (u, w) in enumerate(g.edges):
        for src in (u, w):
            m = s.get_message(e, src)
            assert np.allclose(m, m.conj().T, atol=1e-6)
            assert abs(np.linalg.norm(m) - 1) < 1e-5
            assert np.linalg.eigvalsh(m).min() > -1e-5
    assert np.all(np.abs(s.expect_z_all()) <= 1 + 1e-6)
    s.close()


def test_chi_one_is_a_product_state(tnlib):
    g = OG.ring(12)
    o = OB.run(g, 1, 0.5, 3)
    s = make(tnlib, g, 1)
    s.apply_floquet(0.5, 3)
    assert np.abs(s.expect_z_all() - o.all_z()).max() < Z_TOL
    s.close()


def test_stats_report_bp_iterations(tnlib):
    g = OG.ring(12)
    s = make(tnlib, g, 8)
    s.apply_floquet(0.8, 5)
    st = s.stats()
    assert st["steps_done"] == 5
    assert st["bp_iters_total"] >= 5
    # FP32 messages stop improving near 1e-7: the sweep ends at that floor
    assert st["bp_residual_last"] < 2e-6
    assert st["kernel_launches"] > 0
    assert 0 <= st["discarded_max"] < 1
    s.close()
