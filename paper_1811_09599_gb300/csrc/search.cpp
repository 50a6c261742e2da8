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
//      r - alpha * max(a, b) + beta * log2 runs(D) + tau * gumbel
//    (log2 sizes: result r, inputs a, b; D the cuts the result depends on,
//    runs(D) how often the step reruns per bitstring, below), plus a large
//    penalty when r exceeds the size limit, so that such a step is taken only
//    when nothing else is left; ties are broken by the work 2^(a + b - s) and
//    the larger tensor keeps its id (dst).  Tensors sharing no bond are
//    joined only when no connected pair is left.  Trial 0 is deterministic
//    (alpha = 1, beta = tau = 0: least growth of the larger operand); the
//    others draw alpha in [0, 1.5] and tau in [0, 1], and every odd one beta
//    in [0, 2] (steps that rerun per path are put off), from a SplitMix64
//    stream.  The best trial has the smallest excess of its largest tensor
//    over the limit, then the least work.
//  * cuts: beam search by the number of new cuts.  The kCutBeam best sets
//    with k new cuts that still exceed the limit are extended by every bond
//    not yet cut (k + 1), and by every pair of bonds whose CZ projector
//    halves share a diagonal stretch of one qubit (k + 2; their bits are
//    tied: the pair adds the paths of one cut and removes two bonds, which
//    neither does alone), up to max_new.  The result is the best set
//    evaluated (same ranking), which then gets an ordering search with four
//    times the trials.
//  * work model: a step depending on cuts D runs once per change of those
//    cuts along the executor's path order (ascending slice ids, first cut
//    most significant, paths that vanish identically skipped), 2^(a + b - s)
//    complex MACs each -- the executor's reuse rule.  With every path kept
//    that is prod_{c <= max D} 2^{K_c} runs per bitstring; otherwise the
//    changes are counted along the listed nonzero paths.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <atomic>
#include <iterator>
#include <map>
#include <thread>
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

bool valid_cuts(const SearchNet& net, const std::vector<int>& cuts) {
  if (cuts.size() > 64) return false;
  std::vector<char> seen(net.edges.size(), 0);
  for (int e : cuts) {
    if (e < 0 || e >= int(net.edges.size()) || seen[size_t(e)]) return false;
    seen[size_t(e)] = 1;
  }
  return true;
}

// Runs of a step per bitstring by the cuts it depends on (work model above).
class RunModel {
 public:
  RunModel(const SearchNet& net, const std::vector<int>& cuts) : prefix_(cuts.size() + 1, 1.0) {
    for (size_t c = 0; c < cuts.size(); ++c)
      prefix_[c + 1] = prefix_[c] * std::ldexp(1.0, net.bits[size_t(cuts[c])]);
    n_slices = prefix_.back();
    n_nonzero = n_slices;
    const SliceZeros zeros(net.lines, net.bits, cuts);
    if (!zeros.any()) return;
    n_nonzero = zeros.n_nonzero();
    std::vector<int64_t> ids;
    if (!zeros.list(&ids, kMaxListed)) return;   // too many: count as if all were kept
    vals_.resize(ids.size());
    for (size_t k = 0; k < ids.size(); ++k) {
      int64_t v = ids[k];
      vals_[k].resize(cuts.size());
      for (size_t c = cuts.size(); c-- > 0;) {
        const int bits = net.bits[size_t(cuts[c])];
        vals_[k][c] = v & ((int64_t(1) << bits) - 1);
        v >>= bits;
      }
    }
  }

  double runs(uint64_t dep) {
    if (!dep) return 1.0;
    if (vals_.empty()) {
      int hi = 63;
      while (!((dep >> hi) & 1)) --hi;
      return prefix_[size_t(hi) + 1];
    }
    auto it = memo_.find(dep);
    if (it != memo_.end()) return it->second;
    double r = 0;
    for (size_t k = 0; k < vals_.size(); ++k) {
      bool changed = k == 0;
      for (size_t c = 0; !changed && c < vals_[k].size(); ++c)
        changed = ((dep >> c) & 1) && vals_[k][c] != vals_[k - 1][c];
      r += changed ? 1.0 : 0.0;
    }
    memo_[dep] = r;
    return r;
  }

  double n_slices = 1, n_nonzero = 1;

 private:
  static constexpr int64_t kMaxListed = int64_t(1) << 18;
  std::vector<double> prefix_;
  std::vector<std::vector<int64_t>> vals_;   // listed nonzero paths, value per cut
  std::map<uint64_t, double> memo_;
};

uint64_t splitmix(uint64_t& x) {
  x += 0x9E3779B97F4A7C15ull;
  uint64_t z = x;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double uniform01(uint64_t& x) { return (double(splitmix(x) >> 11) + 0.5) * 0x1.0p-53; }

// One greedy pass with parameters (alpha, beta, tau) and noise stream `rng`;
// results above 2^log2_limit entries are taken only when nothing else is left.
bool greedy_pass(const SearchNet& net, const std::vector<int>& cuts, RunModel& model, double alpha, double beta,
                 double tau, double log2_limit, uint64_t rng, SearchResult* out) {
  const int n = net.n, E = int(net.edges.size());
  if (n < 1) return false;
  std::vector<int> cut_idx(size_t(E), -1);
  for (size_t c = 0; c < cuts.size(); ++c) cut_idx[size_t(cuts[c])] = int(c);
  std::vector<int> leg_bits(size_t(E + n), 1);
  for (int e = 0; e < E; ++e) leg_bits[size_t(e)] = net.bits[size_t(e)];
  auto runs_of = [&](uint64_t dep) { return model.runs(dep); };
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
        if (beta > 0) key += beta * std::log2(runs_of(t[size_t(a)].dep | t[size_t(b)].dep));
        if (double(rr) > log2_limit) key += 1e6;
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
  r.n_slices = model.n_slices;
  r.n_nonzero = model.n_nonzero;
  *out = std::move(r);
  return true;
}

constexpr int kCutBeam = 3;   // cut sets kept per level of the cut search

bool better_result(const SearchResult& x, const SearchResult& y, double log2_limit) {
  const double ox = std::max(0.0, x.log2_max - log2_limit), oy = std::max(0.0, y.log2_max - log2_limit);
  return ox < oy || (ox == oy && x.cmacs < y.cmacs);
}

}  // namespace

bool search_greedy_order(const SearchNet& net, const std::vector<int>& cuts, SearchResult* out, int trials,
                         double log2_limit, uint64_t seed) {
  if (!valid_cuts(net, cuts)) return false;
  RunModel model(net, cuts);
  SearchResult best;
  bool have = false;
  uint64_t x = seed;
  for (int i = 0; i < std::max(1, trials); ++i) {
    const double alpha = i == 0 ? 1.0 : 1.5 * uniform01(x);
    const double tau = i == 0 ? 0.0 : uniform01(x);
    const double beta = (i % 2 == 1) ? 2.0 * uniform01(x) : 0.0;   // odd passes weigh reuse
    SearchResult r;
    if (!greedy_pass(net, cuts, model, alpha, beta, tau, log2_limit, splitmix(x), &r)) return false;
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
  struct State {
    std::vector<int> cuts;
    SearchResult r;
  };
  // moves: one bond, or two bonds whose CZ projector halves share a diagonal
  // stretch of a qubit (their bits are tied, so cutting both adds the paths
  // of one cut while removing two bonds)
  std::vector<std::vector<int>> moves;
  for (int e = 0; e < int(net.edges.size()); ++e)
    if (net.bits[size_t(e)] > 0) moves.push_back({e});
  {
    std::vector<std::pair<int, int>> pairs;
    for (const auto& line : net.lines) {
      std::vector<int> stretch;
      auto flush = [&]() {
        std::sort(stretch.begin(), stretch.end());
        stretch.erase(std::unique(stretch.begin(), stretch.end()), stretch.end());
        for (size_t i = 0; i < stretch.size(); ++i)
          for (size_t j = i + 1; j < stretch.size(); ++j) pairs.push_back({stretch[i], stretch[j]});
        stretch.clear();
      };
      for (const ProjEvent& ev : line) {
        if (ev.edge < 0)
          flush();
        else
          stretch.push_back(ev.edge);
      }
      flush();
    }
    std::sort(pairs.begin(), pairs.end());
    pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
    for (const auto& [a, b] : pairs) moves.push_back({a, b});
  }
  // layers by the number of new cuts: the kCutBeam best states of a layer
  // that do not fit yet are extended by every move within the budget (a
  // pair lands two layers further); every evaluated set competes for the
  // result, so a tied pair that fits with less work than a shallower set
  // is still found
  const size_t base = cuts.size();
  std::vector<std::vector<State>> layer(size_t(max_new) + 1);
  std::vector<std::vector<int>> seen;   // sorted new cuts of every evaluated set
  State best;
  best.cuts = cuts;
  if (!search_greedy_order(net, cuts, &best.r, trials, log2_limit, seed)) return false;
  if (best.r.log2_max > log2_limit && max_new > 0) layer[0].push_back(best);
  for (int k = 0; k < max_new; ++k) {
    std::vector<State>& cur = layer[size_t(k)];
    std::stable_sort(cur.begin(), cur.end(),
                     [&](const State& x, const State& y) { return better_result(x.r, y.r, log2_limit); });
    if (cur.size() > size_t(kCutBeam)) cur.resize(size_t(kCutBeam));
    // candidate sets of this layer, in a fixed order
    std::vector<State> cand;
    for (const State& st : cur) {
      for (const std::vector<int>& mv : moves) {
        if (k + int(mv.size()) > max_new) continue;
        bool taken = false;
        for (int e : mv) taken = taken || std::find(st.cuts.begin(), st.cuts.end(), e) != st.cuts.end();
        if (taken) continue;
        State c;
        c.cuts = st.cuts;
        c.cuts.insert(c.cuts.end(), mv.begin(), mv.end());
        std::vector<int> key(c.cuts.begin() + long(base), c.cuts.end());
        std::sort(key.begin(), key.end());
        if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
        seen.push_back(std::move(key));
        cand.push_back(std::move(c));
      }
    }
    // ordering searches of the candidates on the host cores (independent:
    // each builds its own work model); results are then taken in the
    // fixed order, so the outcome does not depend on the threads
    std::vector<char> ok(cand.size(), 0);
    std::atomic<size_t> next_i{0};
    auto worker = [&]() {
      for (size_t i = next_i++; i < cand.size(); i = next_i++) {
        try {
          ok[i] = search_greedy_order(net, cand[i].cuts, &cand[i].r, trials, log2_limit, seed) ? 1 : 0;
        } catch (...) {
          ok[i] = 0;
        }
      }
    };
    const size_t n_threads =
        std::min<size_t>(cand.size(), std::max<unsigned>(1, std::min<unsigned>(32, std::thread::hardware_concurrency())));
    std::vector<std::thread> pool;
    pool.reserve(n_threads);
    for (size_t t = 1; t < n_threads; ++t) {
      try {
        pool.emplace_back(worker);
      } catch (...) {   // no more threads: the ones started (and this one) finish the work
        break;
      }
    }
    worker();
    for (std::thread& th : pool) th.join();
    for (size_t i = 0; i < cand.size(); ++i) {
      if (!ok[i]) continue;
      State& c = cand[i];
      const size_t k2 = c.cuts.size() - base;
      if (better_result(c.r, best.r, log2_limit)) best = c;
      if (c.r.log2_max > log2_limit) layer[k2].push_back(std::move(c));
    }
    cur.clear();
  }
  // the chosen cut set gets a longer ordering search of its own
  SearchResult polished;
  if (search_greedy_order(net, best.cuts, &polished, 4 * std::max(1, trials), log2_limit,
                          seed ^ 0x5851F42D4C957F2Dull) &&
      better_result(polished, best.r, log2_limit))
    best.r = std::move(polished);
  const bool fits = best.r.log2_max <= log2_limit;
  *cuts_out = best.cuts;
  *out = std::move(best.r);
  return fits;
}

}  // namespace qflex
