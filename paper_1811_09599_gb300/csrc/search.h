// Contraction-ordering and cut search (host code, search.cpp).
#pragma once

#include <cstdint>
#include <utility>
#include <vector>

#include "slices.h"

namespace qflex {

struct SearchNet {
  int n = 0;                                 // qubits = initial tensors
  std::vector<std::pair<int, int>> edges;    // lattice bonds (qubit pairs)
  std::vector<int> bits;                     // bond bits per edge (0: no gate on it)
  std::vector<char> open;                    // per qubit: output leg kept open (tile)
  ProjLines lines;                           // per qubit: CZ projector halves (slices.h);
                                             // empty: every path is counted
};

struct SearchResult {
  std::vector<int32_t> steps;   // (dst, src) pairs, n - 1 of them
  double log2_max = 0;          // log2 entries of the largest tensor (inputs included)
  double cmacs = 0;             // complex MACs of one bitstring over all slices, with reuse
  double n_slices = 1;
  double n_nonzero = 1;         // paths that do not vanish identically
};

// Best of `trials` randomized greedy orderings of the network with `cuts`
// (edge ids, first most significant) removed, ranked by the excess of the
// largest tensor over 2^log2_limit, then by work; false on an invalid network.
bool search_greedy_order(const SearchNet& net, const std::vector<int>& cuts, SearchResult* out, int trials = 1,
                         double log2_limit = 1e300, uint64_t seed = 0);

// Adds up to max_new cuts to `cuts` (beam search) until the ordering's largest tensor has
// at most 2^log2_limit entries; returns whether it fits.
bool search_cuts(const SearchNet& net, std::vector<int> cuts, int max_new, double log2_limit,
                 std::vector<int>* cuts_out, SearchResult* out, int trials = 1, uint64_t seed = 0);

}  // namespace qflex
