"""Write the FP64 oracle's <Z_v> for the batched 64-instance workload.

The workload (workloads.batched_jobs, seed 20230626): 64 heavy-hex instances,
sizes 27, 65, 127, 433 cycled, chi drawn from {8, 16, 32, 64}, theta_h drawn
uniformly from [0, pi/2], 10 Floquet steps each (Eq. 1: RX(theta_h) on every
qubit, then exp(+i pi/4 Z Z) on every edge by the simple update of Methods
"The simple update procedure", then BP to convergence with tolerance 1e-10,
Methods "Belief propagation on a tensor network state").

The oracle runs every instance whose cost stays within about a minute on one
core: all instances with chi <= 16, those with chi = 32 and at most 127
qubits, and those with chi = 64 and 27 qubits.  Per instance the file records
its index, size, chi, theta, steps, the smallest relative truncation gap
(sigma_chi - sigma_chi+1) / sigma_1 the oracle logged, and <Z_v> for every
qubit.  Graphs: the 27-qubit patch is qubits 0..26 of the 127-qubit layout;
65, 127 and 433 qubits are the heavy-hex layouts of 5 x 11, 7 x 15 and 13 x 27
(oracle/graph.py).

This script calls only oracle/ and writes tests/golden/batched64_oracle.txt
(a few minutes on 8 cores):

    python tests/golden/make_batched64_golden.py
"""
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "batched64_oracle.txt")
STEPS = 10


def covered(size, chi):
    return chi <= 16 or (chi == 32 and size <= 127) or (chi == 64 and size == 27)


def graph_of(size):
    from oracle import graph as OG
    return {27: OG.falcon27_patch, 65: lambda: OG.heavy_hex(5, 11), 127: OG.eagle127,
            433: lambda: OG.heavy_hex(13, 27)}[size]()


def run_one(job):
    i, size, chi, theta, steps = job
    from oracle import bptn as OB
    o = OB.run(graph_of(size), chi, theta, steps)
    return i, size, chi, theta, steps, float(o.min_gap), [float(z) for z in o.all_z()]


def main():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    from workloads import batched_jobs
    jobs = [(i, size, chi, theta, steps) for i, (size, chi, theta, steps)
            in enumerate(batched_jobs(n=64)) if covered(size, chi)]
    assert all(j[4] == STEPS for j in jobs)
    # most expensive first, so that the pool ends together
    jobs.sort(key=lambda j: -(j[1] * j[2] ** 4))
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(8, os.cpu_count() or 1)) as pool:
        res = sorted(pool.map(run_one, jobs, chunksize=1))
    lines = [
        "# FP64 oracle (oracle/bptn.py) <Z_v> for the batched 64-instance workload",
        "# (workloads.batched_jobs, seed 20230626), 10 Floquet steps, start |0...0>, BP tol 1e-10.",
        "# Written by tests/golden/make_batched64_golden.py, which calls only oracle/.",
        "# Eq. 1 (Floquet step), Methods 'The simple update procedure' and 'Belief propagation",
        "# on a tensor network state'.  Rows: 'inst i size n chi c theta t steps s min_gap g',",
        "# then 'Z i <Z_0> .. <Z_n-1>'.",
    ]
    for i, size, chi, theta, steps, gap, z in res:
        lines.append("inst %d size %d chi %d theta %r steps %d min_gap %r"
                     % (i, size, chi, theta, steps, gap))
        lines.append("Z %d " % i + " ".join(repr(x) for x in z))
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", OUT, len(res), "instances")


if __name__ == "__main__":
    main()
