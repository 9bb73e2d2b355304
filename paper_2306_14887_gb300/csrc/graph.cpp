// Host-side graph layer: heavy-hex generator, validation, edge colouring and
// Pauli-string propagation through the Clifford step U(pi/2).
//
// The heavy-hex rule reproduces the IBM Eagle layout of the paper's Fig.
// "heavyhexdiagram" (127 qubits, dangling qubits 13 and 113) and its printed
// weight-10 string (section "Measuring expectation values").
#include "graph.h"

#include <algorithm>
#include <map>
#include <set>
#include <string>

namespace tnbp {

bool heavy_hex(int rows, int cols, HostGraph* out, std::string* why) {
  if (rows < 1 || rows % 2 == 0 || cols < 3 || cols % 4 != 3) {
    *why = "heavy-hex needs odd rows >= 1 and cols = 3 (mod 4)";
    return false;
  }
  std::map<std::pair<int, int>, int> site, bridge;
  int next = 0;
  for (int r = 0; r < rows; ++r) {
    for (int c = 0; c < cols; ++c) {
      if ((r == 0 && c == cols - 1) || (r == rows - 1 && c == 0)) continue;
      site[{r, c}] = next++;
    }
    if (r + 1 < rows)
      for (int c = (r % 2 == 0) ? 0 : 2; c < cols; c += 4) bridge[{r, c}] = next++;
  }
  static const int kEven[4] = {0, 1, 2, 1};
  static const int kOdd[4] = {1, 0, 1, 2};
  struct E { int a, b, col; };
  std::vector<E> es;
  for (int r = 0; r < rows; ++r) {
    for (int c = 0; c + 1 < cols; ++c) {
      auto i = site.find({r, c}), j = site.find({r, c + 1});
      if (i != site.end() && j != site.end())
        es.push_back({i->second, j->second, (r % 2 == 0 ? kEven : kOdd)[c % 4]});
    }
    if (r + 1 < rows)
      for (int c = (r % 2 == 0) ? 0 : 2; c < cols; c += 4) {
        int b = bridge[{r, c}];
        es.push_back({site[{r, c}], b, 2});
        es.push_back({b, site[{r + 1, c}], 0});
      }
  }
  for (auto& e : es)
    if (e.a > e.b) std::swap(e.a, e.b);
  std::sort(es.begin(), es.end(), [](const E& x, const E& y) {
    return x.a != y.a ? x.a < y.a : x.b < y.b;
  });
  out->n = next;
  out->eu.clear();
  out->ew.clear();
  out->colour.clear();
  for (auto& e : es) {
    out->eu.push_back(e.a);
    out->ew.push_back(e.b);
    out->colour.push_back(e.col);
  }
  return true;
}

bool build_graph(int n, int m, const int32_t* edges, const uint8_t* colour, HostGraph* g,
                 std::string* why) {
  if (n < 1 || m < 1 || edges == nullptr) {
    *why = "graph needs n_vertices >= 1, n_edges >= 1 and an edge array";
    return false;
  }
  g->n = n;
  g->eu.assign(m, 0);
  g->ew.assign(m, 0);
  g->colour.assign(m, 0);
  std::set<std::pair<int, int>> seen;
  for (int e = 0; e < m; ++e) {
    int a = edges[2 * e], b = edges[2 * e + 1];
    if (a < 0 || b < 0 || a >= n || b >= n) {
      *why = "edge " + std::to_string(e) + " has an endpoint out of range";
      return false;
    }
    if (a == b) {
      *why = "edge " + std::to_string(e) + " is a self-loop";
      return false;
    }
    if (!seen.insert({std::min(a, b), std::max(a, b)}).second) {
      *why = "edge " + std::to_string(e) + " repeats an earlier edge";
      return false;
    }
    g->eu[e] = a;
    g->ew[e] = b;
  }
  g->legs.assign(n, {});
  for (int e = 0; e < m; ++e) {
    g->legs[g->eu[e]].push_back(e);
    g->legs[g->ew[e]].push_back(e);
  }
  for (int v = 0; v < n; ++v) {
    int d = (int)g->legs[v].size();
    if (d < 1 || d > 3) {
      *why = "vertex " + std::to_string(v) + " has degree " + std::to_string(d) +
             " (supported: 1..3)";
      return false;
    }
  }
  if (colour) {
    for (int e = 0; e < m; ++e) g->colour[e] = colour[e];
  } else {
    // first-fit proper edge colouring
    std::vector<std::set<int>> used(n);
    for (int e = 0; e < m; ++e) {
      int c = 0;
      while (used[g->eu[e]].count(c) || used[g->ew[e]].count(c)) ++c;
      used[g->eu[e]].insert(c);
      used[g->ew[e]].insert(c);
      g->colour[e] = c;
    }
  }
  for (int v = 0; v < n; ++v) {
    std::set<int> cs;
    for (int e : g->legs[v])
      if (!cs.insert(g->colour[e]).second) {
        *why = "colouring is not proper at vertex " + std::to_string(v);
        return false;
      }
  }
  std::map<int, std::vector<int>> by;
  for (int e = 0; e < m; ++e) by[g->colour[e]].push_back(e);
  g->layers.clear();
  for (auto& kv : by) g->layers.push_back(kv.second);
  return true;
}

// ------------------------------------------------------------------------
// Pauli strings under conjugation by the Clifford gates of U(pi/2).
//
// Codes: 0 = I, 1 = X, 2 = Y, 3 = Z; the phase is i^phase.
// Single-qubit products used by the ZZ conjugation: P * Z for P in {I,X,Y,Z}
// is {Z, -iY, iX, I}.
// RX(pi/2) P RX(pi/2)^dagger: X -> X, Y -> Z, Z -> -Y (from
// exp(-i t X/2) P exp(i t X/2) = cos t P + i sin t P X for P anticommuting with X).
// exp(+-i pi/4 A) P exp(-+i pi/4 A) = -+i P A for P anticommuting with A = Z_a Z_b.
// ------------------------------------------------------------------------
static void mul_z(uint8_t* p, int* phase) {
  switch (*p) {
    case 0: *p = 3; break;
    case 1: *p = 2; *phase += 3; break;  // X Z = -i Y
    case 2: *p = 1; *phase += 1; break;  // Y Z = +i X
    case 3: *p = 0; break;
  }
}

static void conj_zz(PauliString* s, int a, int b, int sign) {
  uint8_t& pa = s->ops[a];
  uint8_t& pb = s->ops[b];
  int anti = ((pa == 1 || pa == 2) ? 1 : 0) ^ ((pb == 1 || pb == 2) ? 1 : 0);
  if (!anti) return;
  mul_z(&pa, &s->phase);
  mul_z(&pb, &s->phase);
  s->phase += (sign > 0) ? 3 : 1;  // sign +1: -i ; sign -1: +i
  s->phase &= 3;
}

static void conj_rx(PauliString* s, int q, int dagger) {
  uint8_t& p = s->ops[q];
  if (p == 2) {           // Y -> Z (forward), -Z (dagger)
    p = 3;
    if (dagger) s->phase = (s->phase + 2) & 3;
  } else if (p == 3) {    // Z -> -Y (forward), Y (dagger)
    p = 2;
    if (!dagger) s->phase = (s->phase + 2) & 3;
  }
}

void clifford_step(PauliString* s, const HostGraph& g, bool dagger) {
  const int m = (int)g.eu.size();
  if (!dagger) {  // U P U^dagger with U = ZZ * RX
    for (int q = 0; q < g.n; ++q) conj_rx(s, q, 0);
    for (int e = 0; e < m; ++e) conj_zz(s, g.eu[e], g.ew[e], +1);
  } else {        // U^dagger P U
    for (int e = 0; e < m; ++e) conj_zz(s, g.eu[e], g.ew[e], -1);
    for (int q = 0; q < g.n; ++q) conj_rx(s, q, 1);
  }
}

bool reduce_to_single_z(const PauliString& in, const HostGraph& g, int max_steps,
                        int* site, int* nprime, int* sign) {
  PauliString s = in;
  for (int k = 0; k <= max_steps; ++k) {
    int nz = 0, where = -1, other = 0;
    for (int q = 0; q < g.n; ++q) {
      if (s.ops[q] == 3) { ++nz; where = q; }
      else if (s.ops[q] != 0) ++other;
    }
    if (nz == 1 && other == 0 && (s.phase & 1) == 0) {
      *site = where;
      *nprime = k;
      *sign = (s.phase == 0) ? 1 : -1;
      return true;
    }
    clifford_step(&s, g, true);
  }
  return false;
}

}  // namespace tnbp
