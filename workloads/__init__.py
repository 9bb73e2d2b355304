"""Seeded synthetic inputs shared by the tests, the bench and the oracle legs.

This module holds no arithmetic of the method: only random draws, angle grids
and workload descriptions (sizes, chi, step counts).  Both the CUDA path and
the CPU oracle receive these inputs; neither side's algorithm lives here.

Workloads (all synthetic; the paper measures on no public dataset):

* ring12: one heavy hexagon (12-qubit ring), chi = 8, 5 steps,
  theta_h in {0, 0.3, pi/4, 0.8, pi/2}, BP tol 1e-10.
* eagle127: the 127-qubit heavy-hex layout, chi in {16, 32, 64}, 5..20 steps,
  theta_h = 16 uniform values in [0, pi/2] (endpoints included).
* batched: 64 instances, sizes {27, 65, 127, 433} cycled, chi from
  {8, 16, 32, 64} and theta_h ~ U[0, pi/2] drawn with seed 20230626, 10 steps.
* cell5: the periodic 5-site cell, chi in {128, 256}, 50 steps,
  theta_h in {0.4, 0.7, 1.0}.
* serving: Poisson arrivals at 200 jobs/s (seed 7), 2000 jobs, sizes
  {27, 127, 433, 1121}, chi in {16, 32, 64, 128}, theta_h ~ U[0, pi/2],
  steps ~ U{5..20}.
"""
from __future__ import annotations

import numpy as np

THETA_SMALL = (0.0, 0.3, np.pi / 4, 0.8, np.pi / 2)
THETA_SWEEP = tuple(np.linspace(0.0, np.pi / 2, 16))

HEAVY_HEX_SIZES = {27: None, 65: (5, 11), 127: (7, 15), 433: (13, 27), 1121: (21, 43)}


def rng(seed):
    return np.random.default_rng(seed)


def random_site_tensor(r, degree, dims):
    """Complex Gaussian tensor of shape (2, dims[0], .., dims[degree-1])."""
    shape = (2,) + tuple(int(d) for d in dims[:degree])
    return (r.standard_normal(shape) + 1j * r.standard_normal(shape)) / np.sqrt(2)


def random_psd(r, d, rank=None):
    """Random Hermitian positive semi-definite d x d matrix of given rank,
    scaled to unit Frobenius norm."""
    k = d if rank is None else rank
    a = r.standard_normal((d, k)) + 1j * r.standard_normal((d, k))
    m = a @ a.conj().T
    return m / np.linalg.norm(m)


def random_state(degrees, edges, chi, seed):
    """Random site tensors (all bonds of dimension chi) and random PSD messages
    for every directed edge.  ``edges`` is a list of (u, w); legs of a vertex are
    its incident edges in increasing edge id.  Returns (tensors, messages) with
    messages keyed by (src, edge_id)."""
    r = rng(seed)
    tensors = [random_site_tensor(r, d, [chi] * d) for d in degrees]
    msgs = {}
    for e, (u, w) in enumerate(edges):
        msgs[(u, e)] = random_psd(r, chi)
        msgs[(w, e)] = random_psd(r, chi)
    return tensors, msgs


def batched_jobs(n=64, seed=20230626):
    """The batched workload: (size, chi, theta, steps) per instance."""
    r = rng(seed)
    sizes = [27, 65, 127, 433]
    chis = r.choice([8, 16, 32, 64], size=n)
    thetas = r.uniform(0.0, np.pi / 2, size=n)
    return [(sizes[i % 4], int(chis[i]), float(thetas[i]), 10) for i in range(n)]


def serving_jobs(n=2000, rate=200.0, seed=7):
    """The serving workload: (arrival_s, size, chi, theta, steps) per job."""
    r = rng(seed)
    gaps = r.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps)
    sizes = r.choice([27, 127, 433, 1121], size=n)
    chis = r.choice([16, 32, 64, 128], size=n)
    thetas = r.uniform(0.0, np.pi / 2, size=n)
    steps = r.integers(5, 21, size=n)
    return [(float(t[i]), int(sizes[i]), int(chis[i]), float(thetas[i]), int(steps[i]))
            for i in range(n)]


def serving_oracle_sample(n_jobs=200, frac=0.02, seed=11):
    """Indices of the seeded sample of the first `n_jobs` serving jobs that the
    FP64 oracle checks: frac * n_jobs jobs (at least 1) drawn without
    replacement among those with at most 127 qubits and chi at most 64."""
    jobs = serving_jobs(n=2000)[:n_jobs]
    elig = [i for i, j in enumerate(jobs) if j[1] <= 127 and j[2] <= 64]
    k = max(1, int(round(frac * n_jobs)))
    return sorted(int(i) for i in rng(seed).choice(elig, size=min(k, len(elig)), replace=False))

