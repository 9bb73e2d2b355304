"""Lattices for the oracle (test infrastructure; see ``oracle/__init__``).

The heavy-hex lattice is a hexagonal lattice with one extra qubit placed on
every edge (Model and Ansatz, Fig. "heavyhexdiagram"); the IBM Eagle device is
6 x 3 heavy hexagons plus two dangling qubits, 13 and 113.  The paper does not
print coordinates, so the numbering follows the rule below, which reproduces
the paper's printed weight-10 string (Eq. in "Measuring expectation values")
and the two dangling qubits:

* ``R`` rows (``R`` odd) of ``L`` columns (``L = 3 mod 4``); row 0 has no
  column ``L-1`` and row ``R-1`` has no column 0;
* between rows ``r`` and ``r+1`` one bridge qubit sits at every column
  ``c = 0 (mod 4)`` when ``r`` is even and ``c = 2 (mod 4)`` when ``r`` is odd;
* numbering is row-major, each bridge row numbered right after the row above;
* edges join row neighbours and each bridge to the row qubit above and below.

Edge colouring (three layers of disjoint edges, the order in which the ZZ
gates are applied; the paper leaves it free since the gates commute): row edge
``(r,c)-(r,c+1)`` gets ``[0,1,2,1][c%4]`` on even rows and ``[1,0,1,2][c%4]``
on odd rows; a bridge's upper edge gets 2 and its lower edge 0.

This module is written independently of the library's C++ generator; a test
checks that the two agree.
"""
from __future__ import annotations

from collections import deque

import numpy as np


class Graph:
    """Undirected simple graph with an ordered edge list and an edge colouring."""

    def __init__(self, n, edges, colours, name=""):
        self.n = int(n)
        self.edges = [tuple(int(x) for x in e) for e in edges]
        self.colours = [int(c) for c in colours]
        self.name = name
        assert len(self.colours) == len(self.edges)
        # legs of vertex v: the incident edge ids in increasing order
        self.legs = [[] for _ in range(self.n)]
        for eid, (u, w) in enumerate(self.edges):
            assert u != w
            self.legs[u].append(eid)
            self.legs[w].append(eid)

    def degree(self, v):
        return len(self.legs[v])

    def other(self, eid, v):
        u, w = self.edges[eid]
        return w if u == v else u

    def neighbours(self, v):
        return [self.other(e, v) for e in self.legs[v]]

    def layers(self):
        """Edge ids grouped by colour, colours in increasing order."""
        out = {}
        for eid, c in enumerate(self.colours):
            out.setdefault(c, []).append(eid)
        return [out[c] for c in sorted(out)]

    def ball(self, centres, radius):
        """Vertices within graph distance ``radius`` of any centre (BFS)."""
        dist = {}
        q = deque()
        for c in centres:
            dist[c] = 0
            q.append(c)
        while q:
            v = q.popleft()
            if dist[v] == radius:
                continue
            for w in self.neighbours(v):
                if w not in dist:
                    dist[w] = dist[v] + 1
                    q.append(w)
        return sorted(dist)

    def colouring_is_proper(self):
        for v in range(self.n):
            cs = [self.colours[e] for e in self.legs[v]]
            if len(cs) != len(set(cs)):
                return False
        return True


def heavy_hex(R: int, L: int) -> Graph:
    """Heavy-hex patch by the row/bridge rule in the module docstring."""
    assert R % 2 == 1 and L % 4 == 3, "rule needs R odd and L = 3 mod 4"
    index = {}            # (row, col) -> qubit id
    bridge = {}           # (row, col) -> qubit id of the bridge below row
    nxt = 0
    for r in range(R):
        for c in range(L):
            if (r == 0 and c == L - 1) or (r == R - 1 and c == 0):
                continue
            index[(r, c)] = nxt
            nxt += 1
        if r < R - 1:
            first = 0 if r % 2 == 0 else 2
            for c in range(first, L, 4):
                bridge[(r, c)] = nxt
                nxt += 1
    edges, colours = [], []
    row_even = [0, 1, 2, 1]
    row_odd = [1, 0, 1, 2]
    for r in range(R):
        for c in range(L - 1):
            if (r, c) in index and (r, c + 1) in index:
                edges.append((index[(r, c)], index[(r, c + 1)]))
                colours.append((row_even if r % 2 == 0 else row_odd)[c % 4])
        if r < R - 1:
            first = 0 if r % 2 == 0 else 2
            for c in range(first, L, 4):
                b = bridge[(r, c)]
                edges.append((index[(r, c)], b))
                colours.append(2)
                edges.append((b, index[(r + 1, c)]))
                colours.append(0)
    # sort edges by (min, max) so edge ids do not depend on generation order
    order = sorted(range(len(edges)), key=lambda i: (min(edges[i]), max(edges[i])))
    edges = [tuple(sorted(edges[i])) for i in order]
    colours = [colours[i] for i in order]
    return Graph(nxt, edges, colours, name=f"heavyhex{R}x{L}")


def eagle127() -> Graph:
    """The 127-qubit Eagle layout: 6 x 3 heavy hexagons plus qubits 13 and 113."""
    return heavy_hex(7, 15)


def induced(g: Graph, vertices) -> Graph:
    """Induced subgraph, vertices relabelled 0..k-1 in increasing order."""
    vs = sorted(vertices)
    rel = {v: i for i, v in enumerate(vs)}
    edges, colours = [], []
    for (u, w), c in zip(g.edges, g.colours):
        if u in rel and w in rel:
            edges.append((rel[u], rel[w]))
            colours.append(c)
    return Graph(len(vs), edges, colours, name=f"{g.name}[{len(vs)}]")


def falcon27_patch() -> Graph:
    """Induced subgraph on qubits 0..26 of the 127-qubit numbering (two hexagons)."""
    return induced(eagle127(), range(27))


def ring(n: int = 12) -> Graph:
    """One heavy hexagon: a ring of n qubits, edge (i, i+1 mod n), colour i mod 2."""
    assert n % 2 == 0
    return Graph(n, [(i, (i + 1) % n) for i in range(n)],
                 [i % 2 for i in range(n)], name=f"ring{n}")


def path(n: int) -> Graph:
    """Open chain (a tree), colour i mod 2."""
    return Graph(n, [(i, i + 1) for i in range(n - 1)],
                 [i % 2 for i in range(n - 1)], name=f"path{n}")


def star3_tree() -> Graph:
    """A small tree with a degree-3 centre and three 2-qubit arms (7 qubits)."""
    edges = [(0, 1), (0, 3), (0, 5), (1, 2), (3, 4), (5, 6)]
    colours = [0, 1, 2, 1, 2, 0]
    return Graph(7, edges, colours, name="star7")


def spanning_tree(g: Graph) -> Graph:
    """BFS spanning tree of a connected graph (keeps colours of kept edges)."""
    seen = {0}
    keep = []
    q = deque([0])
    while q:
        v = q.popleft()
        for e in g.legs[v]:
            w = g.other(e, v)
            if w not in seen:
                seen.add(w)
                keep.append(e)
                q.append(w)
    keep.sort()
    return Graph(g.n, [g.edges[e] for e in keep], [g.colours[e] for e in keep],
                 name=f"tree({g.name})")


def periodic_cell() -> Graph:
    """Five-site unit cell of the infinite heavy-hex lattice with periodic bonds.

    Two hexagonal-lattice corners A=0, B=1 and three bond midpoints m1..m3 =
    2, 3, 4; A-m_k has colour k-1 and B-m_k colour k mod 3 (the cell is the
    K_{2,3} multigraph-free graph; BP on it is BP on the infinite lattice,
    "Dynamics of the infinite heavy-hex lattice")."""
    edges = [(0, 2), (0, 3), (0, 4), (1, 2), (1, 3), (1, 4)]
    colours = [0, 1, 2, 1, 2, 0]
    return Graph(5, edges, colours, name="cell5")


def hexagon_patches():
    """Heavy-hex patches of one and two hexagons (12 and 21 qubits) cut from the
    127-qubit layout: the 12-ring around the top-left hexagon and its union with
    the next hexagon to the right."""
    g = eagle127()
    # top-left hexagon: row0 cols 0..4, bridges at col 0 and 4, row1 cols 0..4
    one = [0, 1, 2, 3, 4, 14, 15, 18, 19, 20, 21, 22]
    two = one + [5, 6, 7, 8, 16, 23, 24, 25, 26]
    return induced(g, one), induced(g, two)


def greedy_colouring(n, edges):
    """Proper edge colouring by first-fit (used only for graphs with no rule)."""
    used = [set() for _ in range(n)]
    cols = []
    for u, w in edges:
        c = 0
        while c in used[u] or c in used[w]:
            c += 1
        used[u].add(c)
        used[w].add(c)
        cols.append(c)
    return cols


def degree_histogram(g: Graph):
    return np.bincount([g.degree(v) for v in range(g.n)], minlength=4)
