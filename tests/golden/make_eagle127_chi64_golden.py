"""Write the golden values of the FP64 oracle for the 127-qubit chi = 64 workload.

The workload the library's benchmark runs: the 127-qubit heavy-hex graph
(Eagle layout, rule of oracle/graph.py), bond dimension chi = 64, theta_h =
linspace(0, pi/2, 16)[9] = 0.9424777960769379, start |0...0>, BP tolerance
1e-10.  After 8 and 10 Floquet steps (Eq. 1: RX(theta_h) on every qubit, then
exp(+i pi/4 Z Z) on every edge in the colour layers 0, 1, 2 by the simple
update of Methods "The simple update procedure", then BP to convergence,
Methods "Belief propagation on a tensor network state") the file records

* <Z_v> for every qubit (Eq. "SingleSIte" with the converged messages);
* the normalised kept spectrum S of every edge as its last gate set it (the
  message diag(S) the simple update writes on the gate edge);
* the smallest relative gap (sigma_chi - sigma_chi+1) / sigma_1 of any
  truncation so far, the largest discarded weight and the BP sweep count.

Bonds saturate at chi from step 7 on, so every gate of steps 7-10 truncates.

This script calls only oracle/ and writes tests/golden/eagle127_chi64_theta0.9425.txt
(about 6 minutes on 8 cores):

    python tests/golden/make_eagle127_chi64_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import bptn as OB  # noqa: E402
from oracle import graph as OG  # noqa: E402

OUT = os.path.join(HERE, "eagle127_chi64_theta0.9425.txt")
CHI = 64
THETA = float(np.linspace(0.0, np.pi / 2, 16)[9])
RECORD = (8, 10)


def main():
    g = OG.eagle127()
    st = OB.BPState(g, CHI)
    spectra = {}
    lines = [
        "# FP64 oracle (oracle/bptn.py) on the 127-qubit heavy-hex graph (Eagle layout), chi = 64,",
        "# theta_h = %r (linspace(0, pi/2, 16)[9]), start |0...0>, BP tol 1e-10." % THETA,
        "# Written by tests/golden/make_eagle127_chi64_golden.py, which calls only oracle/.",
        "# Eq. 1 (Floquet step), Methods 'The simple update procedure' and 'Belief propagation",
        "# on a tensor network state'.  Rows: 'step s min_gap g discarded_max d bp_iters i',",
        "# 'Z s <Z_0> .. <Z_126>', 'S s e <S_1> .. <S_64>' (spectrum of edge e set by its last gate).",
    ]
    for step in range(1, max(RECORD) + 1):
        st.apply_rx(THETA)
        n_before = len(st.discarded)
        for layer in g.layers():
            for e in layer:
                st.apply_zz(e, +1)
                v = g.edges[e][0]
                s = np.real(np.diag(st.M[(v, e)])).copy()
                spectra[e] = np.pad(s, (0, CHI - len(s)))
        iters, res = st.bp_converge(1e-10, 1000)
        disc = max(st.discarded[n_before:]) if len(st.discarded) > n_before else 0.0
        print("step %d: bp %d sweeps (residual %.2e), min gap %.3e, discarded max %.3e"
              % (step, iters, res, st.min_gap, disc), flush=True)
        if step in RECORD:
            z = st.all_z()
            lines.append("step %d min_gap %r discarded_max %r bp_iters %d"
                         % (step, float(st.min_gap), float(disc), iters))
            lines.append("Z %d " % step + " ".join(repr(float(x)) for x in z))
            for e in range(len(g.edges)):
                lines.append("S %d %d " % (step, e) + " ".join("%.15e" % x for x in spectra[e]))
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
