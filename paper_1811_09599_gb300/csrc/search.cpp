// Contraction-ordering and cut search (host code).
//
// The paper fixes, for each lattice, a set of cut bonds and a contraction
// order by hand (Methods, "Cutting indexes" and "Contraction of the 3D
// tensor network"; SI A), so that every tensor fits in memory and partial
// contractions that do not depend on a cut are reused across its paths.
// This file searches both automatically:
//
//  * ordering: randomized greedy over the per-slice network (cut bonds
//    removed), best of several trials.  Each step contracts the pair of live
//    tensors sharing a bond with the smallest key
//      r - alpha * max(a, b) + tau * gumbel     (log2 sizes: result r,
//                                                inputs a, b)
//    ties broken by the work 2^(a + b - s); the larger tensor keeps its id
//    (dst).  Tensors sharing no bond are joined only when no connected pair
//    is left.  Trial 0 is deterministic (alpha = 1, tau = 0: least growth of
//    the larger operand); the others draw alpha in [0, 1.5] and tau in
//    [0, 1] from a SplitMix64 stream.  The best trial has the smallest
//    excess of its largest tensor over the limit, then the least work.
//  * cuts: while the largest tensor of the greedy ordering exceeds the
//    limit, add the bond whose cut gives the smallest largest tensor, ties
//    broken by the total work of one bitstring.
//  * work model: a step depending on cuts D runs once per change of those
//    cuts in mixed-radix slice order (first cut most significant), i.e.
//    prod_{c <= max D} 2^{K_c} times per bitstring, 2^(a + b - s) complex
//    MACs each -- the executor's reuse rule.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <iterator>
#include <utility>
#include <vector>

#include "search.h"

namespace qflex {
namespace {

struct Tensor {
  std::vector<int> legs;   // sorted: edge ids, or E + q for qubit q's open output leg
  int bits = 0;            // log2 entries
  uint64_t dep = 0;        // cuts whose values it depends on
};

int shared_bits(const Tensor& a, const Tensor& b, const std::vector<int>& leg_bits) {
  int s = 0;
  size_t i = 0, j = 0;
  while (i < a.legs.size() && j < b.legs.size()) {
    if (a.legs[i] < b.legs[j]) {
      ++i;
    } else if (a.legs[i] > b.legs[j]) {
      ++j;
    } else {
      s += leg_bits[size_t(a.legs[i])];
      ++i;
      ++j;
    }
  }
  return s;
}

Tensor merge(const Tensor& a, const Tensor& b, const std::vector<int>& leg_bits) {
  Tensor r;
  std::set_symmetric_difference(a.legs.begin(), a.legs.end(), b.legs.begin(), b.legs.end(),
                                std::back_inserter(r.legs));
  for (int l : r.legs) r.bits += leg_bits[size_t(l)];
  r.dep = a.dep | b.dep;
  return r;
}

uint64_t splitmix(uint64_t& x) {
  x += 0x9E3779B97F4A7C15ull;
  uint64_t z = x;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double uniform01(uint64_t& x) { return (double(splitmix(x) >> 11) + 0.5) * 0x1.0p-53; }

// One greedy pass with parameters (alpha, tau) and noise stream `rng`.
bool greedy_pass(const SearchNet& net, const std::vector<int>& cuts, double alpha, double tau, uint64_t rng,
                 SearchResult* out) {
  const int n = net.n, E = int(net.edges.size());
  if (n < 1) return false;
  std::vector<int> cut_idx(size_t(E), -1);
  for (size_t c = 0; c < cuts.size(); ++c) {
    if (cuts[c] < 0 || cuts[c] >= E || cut_idx[size_t(cuts[c])] >= 0 || c >= 64) return false;
    cut_idx[size_t(cuts[c])] = int(c);
  }
  std::vector<int> leg_bits(size_t(E + n), 1);
  for (int e = 0; e < E; ++e) leg_bits[size_t(e)] = net.bits[size_t(e)];
  // runs of a step by its dependence mask: the product of the radices of all
  // cuts down to the least significant one it depends on
  std::vector<double> prefix_runs(cuts.size() + 1, 1.0);
  for (size_t c = 0; c < cuts.size(); ++c)
    prefix_runs[c + 1] = prefix_runs[c] * std::ldexp(1.0, net.bits[size_t(cuts[c])]);
  auto runs_of = [&](uint64_t dep) {
    if (!dep) return 1.0;
    int hi = 63;
    while (!((dep >> hi) & 1)) --hi;
    return prefix_runs[size_t(hi) + 1];
  };
  std::vector<Tensor> t(static_cast<size_t>(n));
  std::vector<char> alive(size_t(n), 1);
  SearchResult r;
  for (int e = 0; e < E; ++e) {
    const int c = cut_idx[size_t(e)];
    for (int q : {net.edges[size_t(e)].first, net.edges[size_t(e)].second}) {
      if (q < 0 || q >= n) return false;
      if (net.bits[size_t(e)] == 0) continue;       // no gate on this edge: no bond
      if (c >= 0) {
        t[size_t(q)].dep |= uint64_t(1) << c;
      } else {
        t[size_t(q)].legs.push_back(e);
      }
    }
  }
  for (int q = 0; q < n; ++q) {
    if (net.open[size_t(q)]) t[size_t(q)].legs.push_back(E + q);
    std::sort(t[size_t(q)].legs.begin(), t[size_t(q)].legs.end());
    for (int l : t[size_t(q)].legs) t[size_t(q)].bits += leg_bits[size_t(l)];
    r.log2_max = std::max(r.log2_max, double(t[size_t(q)].bits));
  }
  for (int step = 0; step < n - 1; ++step) {
    int best_a = -1, best_b = -1;
    double best_key = 0, best_work = 0;
    bool best_conn = false;
    for (int a = 0; a < n; ++a) {
      if (!alive[size_t(a)]) continue;
      for (int b = a + 1; b < n; ++b) {
        if (!alive[size_t(b)]) continue;
        const int s = shared_bits(t[size_t(a)], t[size_t(b)], leg_bits);
        const bool conn = s > 0;
        if (best_conn && !conn) continue;
        const int ra = t[size_t(a)].bits, rb = t[size_t(b)].bits;
        const int rr = ra + rb - 2 * s;
        double key = double(rr) - alpha * double(std::max(ra, rb));
        if (tau > 0) key -= tau * std::log(-std::log(uniform01(rng)));
        const double work = std::ldexp(1.0, ra + rb - s);
        const bool better = best_a < 0 || (conn && !best_conn) || key < best_key ||
                            (key == best_key && work < best_work);
        if (better) {
          best_a = a;
          best_b = b;
          best_key = key;
          best_work = work;
          best_conn = conn;
        }
      }
    }
    if (best_a < 0) return false;
    int dst = best_a, src = best_b;
    if (t[size_t(src)].bits > t[size_t(dst)].bits) std::swap(dst, src);
    const int s = shared_bits(t[size_t(dst)], t[size_t(src)], leg_bits);
    Tensor m = merge(t[size_t(dst)], t[size_t(src)], leg_bits);
    r.cmacs += runs_of(m.dep) * std::ldexp(1.0, t[size_t(dst)].bits + t[size_t(src)].bits - s);
    r.log2_max = std::max(r.log2_max, double(m.bits));
    t[size_t(dst)] = std::move(m);
    alive[size_t(src)] = 0;
    r.steps.push_back(dst);
    r.steps.push_back(src);
  }
  r.n_slices = prefix_runs.back();
  *out = std::move(r);
  return true;
}

bool better_result(const SearchResult& x, const SearchResult& y, double log2_limit) {
  const double ox = std::max(0.0, x.log2_max - log2_limit), oy = std::max(0.0, y.log2_max - log2_limit);
  return ox < oy || (ox == oy && x.cmacs < y.cmacs);
}

}  // namespace

bool search_greedy_order(const SearchNet& net, const std::vector<int>& cuts, SearchResult* out, int trials,
                         double log2_limit, uint64_t seed) {
  SearchResult best;
  bool have = false;
  uint64_t x = seed;
  for (int i = 0; i < std::max(1, trials); ++i) {
    const double alpha = i == 0 ? 1.0 : 1.5 * uniform01(x);
    const double tau = i == 0 ? 0.0 : uniform01(x);
    SearchResult r;
    if (!greedy_pass(net, cuts, alpha, tau, splitmix(x), &r)) return false;
    if (!have || better_result(r, best, log2_limit)) {
      best = std::move(r);
      have = true;
    }
  }
  *out = std::move(best);
  return true;
}

bool search_cuts(const SearchNet& net, std::vector<int> cuts, int max_new, double log2_limit,
                 std::vector<int>* cuts_out, SearchResult* out, int trials, uint64_t seed) {
  SearchResult cur;
  if (!search_greedy_order(net, cuts, &cur, trials, log2_limit, seed)) return false;
  for (int added = 0; cur.log2_max > log2_limit && added < max_new; ++added) {
    int best_e = -1;
    SearchResult best;
    for (int e = 0; e < int(net.edges.size()); ++e) {
      if (net.bits[size_t(e)] == 0 || std::find(cuts.begin(), cuts.end(), e) != cuts.end()) continue;
      std::vector<int> trial = cuts;
      trial.push_back(e);
      SearchResult r;
      if (!search_greedy_order(net, trial, &r, trials, log2_limit, seed)) continue;
      if (best_e < 0 || better_result(r, best, log2_limit)) {
        best_e = e;
        best = std::move(r);
      }
    }
    if (best_e < 0) break;
    cuts.push_back(best_e);
    cur = std::move(best);
  }
  const bool fits = cur.log2_max <= log2_limit;
  *cuts_out = cuts;
  *out = std::move(cur);
  return fits;
}

}  // namespace qflex
