// Host-side graph layer of the tnbp library (internal).
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

namespace tnbp {

struct HostGraph {
  int n = 0;
  std::vector<int> eu, ew, colour;        // edge endpoints and colours
  std::vector<std::vector<int>> legs;     // incident edges per vertex, increasing id
  std::vector<std::vector<int>> layers;   // edge ids per colour, colours increasing
  int other(int e, int v) const { return eu[e] == v ? ew[e] : eu[e]; }
  int degree(int v) const { return (int)legs[v].size(); }
  int leg_pos(int v, int e) const {
    for (int i = 0; i < (int)legs[v].size(); ++i)
      if (legs[v][i] == e) return i;
    return -1;
  }
};

bool heavy_hex(int rows, int cols, HostGraph* out, std::string* why);
bool build_graph(int n, int m, const int32_t* edges, const uint8_t* colour, HostGraph* g,
                 std::string* why);

struct PauliString {
  std::vector<uint8_t> ops;  // per qubit: 0 I, 1 X, 2 Y, 3 Z
  int phase = 0;             // i^phase
};

// s <- U s U^dagger (dagger = false) or U^dagger s U (dagger = true), U = U(pi/2).
void clifford_step(PauliString* s, const HostGraph& g, bool dagger);

// Find n' <= max_steps with U^-n' s U^n' = sign * Z_site (so that
// s = sign * U^n' Z_site U^-n').
bool reduce_to_single_z(const PauliString& s, const HostGraph& g, int max_steps, int* site,
                        int* nprime, int* sign);

}  // namespace tnbp
