"""Host-side checks of the C ABI that need no GPU: the library loads and exports
every declared symbol, the C++ lattice generator equals the oracle's, the host
Pauli propagation reproduces the paper's printed string, and argument errors
come back as status codes."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2306_14887_gb300 as tn
from paper_2306_14887_gb300 import build as B
from oracle import clifford as OC
from oracle import graph as OG

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "tnbp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tn_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    L = C.CDLL(tn.LIB_PATH)
    decl = declared_symbols()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(tn.EXPORTS) == decl


def test_version_string():
    assert "sm_103a" in tn.version()


@pytest.mark.parametrize("R,L", [(7, 15), (5, 11), (13, 27), (21, 43)])
def test_cpp_heavy_hex_matches_oracle(R, L):
    n, edges, cols = tn.heavy_hex(R, L)
    g = OG.heavy_hex(R, L)
    assert n == g.n
    assert [tuple(e) for e in edges.tolist()] == g.edges
    assert cols.tolist() == g.colours


def test_heavy_hex_rejects_bad_shape():
    with pytest.raises(tn.TNError) as ei:
        tn.heavy_hex(6, 15)
    assert ei.value.status == -1


def test_cpp_clifford_reduce_printed_string():
    """The paper's weight-10 string is U^5(pi/2) Z_13 U^5(pi/2)^dagger."""
    n, edges, _ = tn.heavy_hex(7, 15)
    ops = {13: "X", 29: "X", 31: "X", 9: "Y", 30: "Y", 8: "Z", 12: "Z", 17: "Z", 28: "Z",
           32: "Z"}
    assert tn.clifford_reduce(n, edges, ops) == (13, 5, 1)
    assert tn.clifford_reduce(n, edges, ops, sign=-1) == (13, 5, -1)


@pytest.mark.parametrize("site,nprime", [(0, 1), (62, 2), (40, 3), (113, 4), (100, 6)])
def test_cpp_clifford_reduce_matches_oracle(site, nprime):
    g = OG.eagle127()
    s = OC.string_from_z(g, site, nprime)
    n, edges, _ = tn.heavy_hex(7, 15)
    got = tn.clifford_reduce(n, edges, s.ops)
    # the smallest n' that reduces the string may be shorter than the one used
    assert got[0] == site
    assert got[1] <= nprime
    assert got[2] == int(s.phase.real) or got[1] < nprime


def test_clifford_reduce_rejects_non_clifford_string():
    n, edges, _ = tn.heavy_hex(7, 15)
    with pytest.raises(tn.TNError) as ei:
        tn.clifford_reduce(n, edges, {0: "X", 126: "X"}, max_steps=4)
    assert ei.value.status == -8


@pytest.mark.parametrize("edges,why", [
    ([(0, 1), (0, 2), (0, 3), (0, 4)], "degree"),
    ([(0, 0), (0, 1)], "self-loop"),
    ([(0, 1), (1, 0)], "repeats"),
    ([(0, 5)], "range"),
])
def test_create_rejects_bad_graph_before_touching_a_device(edges, why):
    n = 5
    with pytest.raises(tn.TNError) as ei:
        tn.footprint_estimate(n, edges, None, 4)
    assert ei.value.status == -1
    assert why in str(ei.value)


def test_footprint_estimate_scales_with_chi():
    n, edges, cols = tn.heavy_hex(7, 15)
    f16 = tn.footprint_estimate(n, edges, cols, 16)
    f32 = tn.footprint_estimate(n, edges, cols, 32)
    # dominated by the 36 degree-3 tensors (chi^3): 8x from 16 to 32
    assert 6 < f32 / f16 < 9
    # four site-tensor-shaped buffers, FP32 planar complex: 4 * 4 * sum chi^d bytes
    sites = 36 * 32 ** 3 + 89 * 32 ** 2 + 2 * 32
    assert f32 >= 16 * 4 * sites


def test_create_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = tn.lib()
    n, edges, cols = tn.heavy_hex(5, 11)
    g, keep = tn._graph_struct(n, edges, cols)
    cfg = tn._config(4, "fp32", 1e-10, 10, 0.0)
    h = C.c_void_p()
    st = L.tn_create(C.byref(g), C.byref(cfg), None, None, C.byref(h))
    assert st == -6
    assert "CUDA" in L.tn_last_error().decode() or "device" in L.tn_last_error().decode()


def test_batch_union_offsets_and_colouring():
    from oracle import graph as OG
    gs = [OG.ring(12), OG.falcon27_patch(), OG.ring(12)]
    n, edges, cols, offs = tn.batch_union([(g.n, g.edges, g.colours) for g in gs])
    assert n == 12 + 27 + 12 and offs == [0, 12, 39]
    assert len(edges) == sum(len(g.edges) for g in gs) and len(cols) == len(edges)
    # components stay disjoint and each keeps a proper colouring
    for g, off in zip(gs, offs):
        sub = [tuple(e) for e in edges if off <= e[0] < off + g.n]
        assert len(sub) == len(g.edges)
        assert all(off <= a < off + g.n and off <= b < off + g.n for a, b in sub)
    seen = {}
    for (a, b), c in zip(edges, cols):
        for v in (a, b):
            assert (v, c) not in seen
            seen[(v, c)] = True


def test_server_rejects_bad_config_before_touching_a_device():
    cfg = tn.tn_server_config()
    cfg.max_slots = 0
    h = tn.C.c_void_p()
    assert tn.lib().tn_server_create(tn.C.byref(cfg), tn.C.byref(h)) == -1
    # an admission policy other than TN_SERVE_FIFO (0) and TN_SERVE_SHORTEST (1)
    cfg.max_slots = 2
    cfg.policy = 7
    assert tn.lib().tn_server_create(tn.C.byref(cfg), tn.C.byref(h)) == -1
    assert not h.value


def test_autotune_and_components_reject_null_handles():
    L = tn.lib()
    n = tn.C.c_size_t()
    assert L.tn_autotune(None, 3, None, 0, tn.C.byref(n)) == -1
    assert L.tn_autotune_apply(None, b"", None) == -1
    nc = tn.C.c_int32()
    assert L.tn_bp_components(None, None, None, None, 0, tn.C.byref(nc)) == -1


def test_chi_extrapolation_matches_least_squares():
    """tn_chi_extrapolate: the least-squares line in 1/chi (host arithmetic)."""
    r = np.random.default_rng(11)
    chis = np.array([16.0, 32.0, 64.0, 128.0])
    vals = r.standard_normal((4, 7))
    a, b, rms = tn.chi_extrapolate(chis, vals)
    X = np.stack([np.ones(4), 1.0 / chis], axis=1)
    coef, *_ = np.linalg.lstsq(X, vals, rcond=None)
    assert np.allclose(a, coef[0], atol=1e-12) and np.allclose(b, coef[1], atol=1e-12)
    assert np.allclose(rms, np.sqrt(((X @ coef - vals) ** 2).mean(axis=0)), atol=1e-12)


def test_chi_extrapolation_recovers_an_exact_line():
    chis = np.array([8.0, 24.0, 500.0])
    vals = np.stack([0.25 + 3.0 / chis, -1.0 + 0.0 / chis], axis=1)
    a, b, rms = tn.chi_extrapolate(chis, vals)
    assert np.allclose(a, [0.25, -1.0], atol=1e-13) and np.allclose(b, [3.0, 0.0], atol=1e-12)
    assert np.all(rms < 1e-13)


@pytest.mark.parametrize("chis,vals", [([16.0], [[1.0]]), ([16.0, 16.0], [[1.0], [2.0]]),
                                       ([0.0, 16.0], [[1.0], [2.0]]),
                                       ([8.0, 16.0], [[1.0], [np.nan]])])
def test_chi_extrapolation_rejects_bad_input(chis, vals):
    with pytest.raises(tn.TNError):
        tn.chi_extrapolate(chis, vals)
