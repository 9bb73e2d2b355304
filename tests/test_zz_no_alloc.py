"""The allocation-free truncation solve against the allocating one.

tn_truncation_solve_noalloc exists for callers that cannot allocate device
memory themselves or let a library do it (their runtime owns the device pool,
or their loop cannot take the synchronisation of cudaMalloc).  It must give
the same results as tn_truncation_solve, call after call, even though every
call reuses one fixed workspace array inside the library.  This file is named
to run last so that a failure here stops a -x run only after everything else.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module")
def tnlib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_14887_gb300 import build
    build.build()
    import paper_2306_14887_gb300 as tn
    return tn


def random_grams(n_edges, chi, rows, seed):
    r = np.random.default_rng(seed)
    gram = np.zeros((n_edges, 2, 2, 2, chi, chi), dtype=np.float32)
    for k in range(n_edges):
        for side in range(2):
            x = r.standard_normal((2, rows, chi)) + 1j * r.standard_normal((2, rows, chi))
            for p in range(2):
                n_p = x[p].T @ x[p].conj()
                gram[k, side, p, 0] = n_p.real
                gram[k, side, p, 1] = n_p.imag
    return gram


def call(fn, g, chi, n_edges, sign):
    import torch
    d = torch.zeros_like(g)
    s = torch.zeros(n_edges * chi, dtype=torch.float64, device=g.device)
    st = fn(C.c_void_p(g.data_ptr()), C.c_void_p(d.data_ptr()), C.c_void_p(s.data_ptr()),
            n_edges, chi, sign, 0.0, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, d.cpu().numpy(), s.cpu().numpy()


def test_noalloc_matches_allocating_solve_twice_in_a_row(tnlib):
    import torch
    L = tnlib.lib()
    cases = [(6, 8, 12, 1, 21), (3, 16, 24, -1, 22)]   # (edges, chi, rows, sign, seed)
    for n_edges, chi, rows, sign, seed in cases:
        g = torch.from_numpy(random_grams(n_edges, chi, rows, seed).reshape(-1)).cuda()
        st_a, d_a, s_a = call(L.tn_truncation_solve, g, chi, n_edges, sign)
        st_b, d_b, s_b = call(L.tn_truncation_solve_noalloc, g, chi, n_edges, sign)
        assert st_a == 0 and st_b == 0, L.tn_last_error().decode()
        np.testing.assert_allclose(s_b, s_a, atol=TOL, rtol=0)
        np.testing.assert_allclose(d_b, d_a, atol=TOL * max(1.0, np.abs(d_a).max()), rtol=0)
        assert s_a.reshape(n_edges, chi)[:, 0].min() > 0


def test_noalloc_rejects_requests_beyond_its_workspace(tnlib):
    import torch
    L = tnlib.lib()
    g = torch.zeros(8, device="cuda")
    st, _, _ = call(L.tn_truncation_solve_noalloc, g, 64, 11, 1)   # 11 edges at chi = 64
    assert st == -1
    msg = L.tn_last_error().decode()
    assert "16777216" in msg and "workspace" in msg


def test_noalloc_recovers_after_a_failed_call(tnlib):
    """The workspace keeps the previous call's contents, error flag included: a
    call whose spectrum is zero (an all-zero Gram) fails with TN_ENUMERIC, and
    the next, valid call on the same array must succeed and match the
    allocating solve."""
    import torch
    L = tnlib.lib()
    n_edges, chi = 4, 8
    zero = torch.zeros(n_edges * 8 * chi * chi, device="cuda")
    st, _, _ = call(L.tn_truncation_solve_noalloc, zero, chi, n_edges, 1)
    assert st == -4   # TN_ENUMERIC
    g = torch.from_numpy(random_grams(n_edges, chi, 12, 23).reshape(-1)).cuda()
    st_a, d_a, s_a = call(L.tn_truncation_solve, g, chi, n_edges, 1)
    st_b, d_b, s_b = call(L.tn_truncation_solve_noalloc, g, chi, n_edges, 1)
    assert st_a == 0 and st_b == 0, L.tn_last_error().decode()
    np.testing.assert_allclose(s_b, s_a, atol=TOL, rtol=0)
    np.testing.assert_allclose(d_b, d_a, atol=TOL * max(1.0, np.abs(d_a).max()), rtol=0)
