"""Write the FP64 oracle's <Z_v> for the seeded sample of the serving stream.

The serving workload (workloads.serving_jobs, seed 7): Poisson arrivals at 200
jobs/s, each a heavy-hex graph of 27, 127, 433 or 1121 qubits, chi from
{16, 32, 64, 128}, theta_h ~ U[0, pi/2] and 5-20 Floquet steps.  Of its first
200 jobs, a seeded 2% sample (workloads.serving_oracle_sample: 4 jobs drawn
among those with at most 127 qubits and chi at most 64) is run by the FP64
oracle from |0...0>: Eq. 1's Floquet step (RX(theta_h) on every qubit, then
exp(+i pi/4 Z Z) on every edge by the simple update of Methods "The simple
update procedure"), BP to tolerance 1e-10 after each step (Methods "Belief
propagation on a tensor network state").  Per job the file records its index,
size, chi, theta, steps, the smallest relative truncation gap the oracle
logged, and <Z_v> for every qubit.  The 27-qubit graph is qubits 0..26 of the
127-qubit layout (oracle/graph.py).

This script calls only oracle/ and writes tests/golden/serving_sample_oracle.txt
(about 10 minutes on 8 cores):

    python tests/golden/make_serving_golden.py
"""
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "serving_sample_oracle.txt")


def run_one(job):
    i, size, chi, theta, steps = job
    from oracle import bptn as OB
    from oracle import graph as OG
    g = OG.falcon27_patch() if size == 27 else OG.eagle127()
    o = OB.run(g, chi, theta, steps)
    return i, size, chi, theta, steps, float(o.min_gap), [float(z) for z in o.all_z()]


def main():
    from workloads import serving_jobs, serving_oracle_sample
    jobs = serving_jobs(n=2000)
    pick = [(i,) + jobs[i][1:] for i in serving_oracle_sample()]
    threads = max(1, (os.cpu_count() or 1) // len(pick))
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = str(threads)
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(pick)) as pool:
        res = sorted(pool.map(run_one, pick, chunksize=1))
    lines = [
        "# FP64 oracle (oracle/bptn.py) <Z_v> for the seeded 2% sample of the first 200 jobs",
        "# of the serving stream (workloads.serving_jobs seed 7, workloads.serving_oracle_sample",
        "# seed 11), start |0...0>, BP tol 1e-10.",
        "# Written by tests/golden/make_serving_golden.py, which calls only oracle/.",
        "# Eq. 1 (Floquet step), Methods 'The simple update procedure' and 'Belief propagation",
        "# on a tensor network state'.  Rows: 'job i size n chi c theta t steps s min_gap g',",
        "# then 'Z i <Z_0> .. <Z_n-1>'.",
    ]
    for i, size, chi, theta, steps, gap, z in res:
        lines.append("job %d size %d chi %d theta %r steps %d min_gap %r"
                     % (i, size, chi, theta, steps, gap))
        lines.append("Z %d " % i + " ".join(repr(x) for x in z))
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", OUT, len(res), "jobs")


if __name__ == "__main__":
    main()
