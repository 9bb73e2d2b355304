"""CPU FP64 oracle for the BP-approximated tensor-network kicked-Ising simulation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import anything
from this package.  The product library never calls it and shares no code with
it: the oracle has its own lattice generator, its own gate algebra and its own
belief-propagation and simple-update steps, all written in plain NumPy
complex128 from the paper (Tindall, Fishman, Stoudenmire, Sels, "Efficient
tensor network simulation of IBM's Eagle kicked Ising experiment",
arXiv:2306.14887).

Modules
-------
graph        heavy-hex lattice generator, 12-ring, trees, periodic 5-site cell,
             edge colouring, graph balls (Fig. "heavyhexdiagram", Eq. 1)
clifford     Pauli-string propagation through U(pi/2) (the extended time
             evolution identity of "Measuring expectation values")
statevector  exact 2^n statevector evolution and a light-cone restriction
             (the exact references of "Results")
bptn         the BP-approximated TNS algorithm itself (Methods: simple update,
             belief propagation, expectation values), FP64

Pins: every function is checked in ``tests/test_oracle_*.py`` against facts the
paper or mathematics fix (the printed weight-10 string, closed forms at the
Clifford points, exactness of BP on trees and for short circuits, brute-force
statevectors), not against itself.
"""
