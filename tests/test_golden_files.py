"""The stored oracle values under tests/golden/ are the oracle's, for the
workloads the generators describe.

Each file is written by a committed script that calls only oracle/.  Here the
files' recorded parameters are checked against the seeded generators
(workloads/), their values against the ranges the physics fixes, and the
cheapest rows are recomputed by the oracle itself (up to the last bits that
BLAS threading may change)."""
import os

import numpy as np
import pytest

from oracle import bptn as OB
from oracle import graph as OG
from workloads import batched_jobs, serving_jobs, serving_oracle_sample

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SIZES = {27: 27, 65: 65, 127: 127, 433: 433}


def _graph(size):
    return {27: OG.falcon27_patch, 65: lambda: OG.heavy_hex(5, 11), 127: OG.eagle127,
            433: lambda: OG.heavy_hex(13, 27)}[size]()


def _read(name, head):
    rows, z = {}, {}
    for line in open(os.path.join(GOLDEN, name)):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == head:
            kv = dict(zip(f[2::2], f[3::2]))
            rows[int(f[1])] = kv
        elif f[0] == "Z":
            z[int(f[1])] = np.array([float(x) for x in f[2:]])
    return rows, z


def test_batched_golden_matches_the_generator():
    rows, z = _read("batched64_oracle.txt", "inst")
    jobs = batched_jobs(n=64)
    assert len(rows) == 49 and set(rows) == set(z)
    for i, kv in rows.items():
        size, chi, theta, steps = jobs[i]
        assert int(kv["size"]) == size and int(kv["chi"]) == chi and int(kv["steps"]) == steps
        assert float(kv["theta"]) == theta
        assert len(z[i]) == size and np.all(np.abs(z[i]) <= 1 + 1e-12)
        assert float(kv["min_gap"]) >= 0.0


@pytest.mark.parametrize("i", [1, 20])
def test_batched_golden_rows_are_the_oracle(i):
    """Two of the cheapest rows (chi = 8, 65 and 27 qubits) recomputed."""
    rows, z = _read("batched64_oracle.txt", "inst")
    kv = rows[i]
    assert int(kv["chi"]) == 8
    o = OB.run(_graph(int(kv["size"])), 8, float(kv["theta"]), int(kv["steps"]))
    assert np.abs(o.all_z() - z[i]).max() < 1e-12


def test_serving_golden_matches_the_generator_and_the_oracle():
    rows, z = _read("serving_sample_oracle.txt", "job")
    pick = serving_oracle_sample()
    assert sorted(rows) == pick and len(pick) == 4
    jobs = serving_jobs(n=2000)
    for i, kv in rows.items():
        _, size, chi, theta, steps = jobs[i]
        assert size <= 127 and chi <= 64
        assert (int(kv["size"]), int(kv["chi"]), float(kv["theta"]), int(kv["steps"])) == \
            (size, chi, theta, steps)
        assert len(z[i]) == size and np.all(np.abs(z[i]) <= 1 + 1e-12)
    # the cheapest job recomputed (27 qubits, chi = 32, 7 steps)
    i = min(rows, key=lambda k: int(rows[k]["size"]) * int(rows[k]["chi"]) ** 4 * int(rows[k]["steps"]))
    kv = rows[i]
    o = OB.run(_graph(int(kv["size"])), int(kv["chi"]), float(kv["theta"]), int(kv["steps"]))
    assert np.abs(o.all_z() - z[i]).max() < 1e-12


def test_headline_golden_structure():
    """127 qubits, chi = 64, steps 8 and 10: 127 values of <Z> per step, one
    normalised kept spectrum of 64 values per edge, decreasing, of unit norm."""
    path = os.path.join(GOLDEN, "eagle127_chi64_theta0.9425.txt")
    z, spec, steps = {}, {}, []
    for line in open(path):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "step":
            steps.append(int(f[1]))
            assert float(f[3]) > 1e-6  # no near-tie: the comparison is element by element
        elif f[0] == "Z":
            z[int(f[1])] = np.array([float(x) for x in f[2:]])
        elif f[0] == "S":
            spec[(int(f[1]), int(f[2]))] = np.array([float(x) for x in f[3:]])
    assert steps == [8, 10]
    for s in steps:
        assert len(z[s]) == 127 and np.all(np.abs(z[s]) <= 1)
        for e in range(144):
            v = spec[(s, e)]
            assert len(v) == 64
            assert np.all(np.diff(v) <= 1e-15) and abs(np.linalg.norm(v) - 1) < 1e-12
