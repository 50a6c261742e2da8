// Paths that vanish identically: the projector rule of slices.h as bit
// classes.  Every bit of a cut value is a node; the projector bits of one
// diagonal stretch are joined (union-find), and those of a first stretch
// are joined with a node standing for the constant 0.  A path is nonzero
// exactly when every class is constant on it (and 0 on the class of the
// constant), so the nonzero paths are the free choices of one bit per class
// not tied to 0.
#include "slices.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace qflex {

SliceZeros::SliceZeros(const ProjLines& lines, const std::vector<int>& edge_bits, const std::vector<int>& cuts) {
  const int E = int(edge_bits.size());
  std::vector<int> cut_of(size_t(E), -1), node_off(cuts.size() + 1, 0);
  for (size_t c = 0; c < cuts.size(); ++c) {
    cut_of[size_t(cuts[c])] = int(c);
    cut_bits_.push_back(edge_bits[size_t(cuts[c])]);
    node_off[c + 1] = node_off[c] + cut_bits_.back();
  }
  const int n_nodes = node_off.back();
  const int zero_node = n_nodes;
  std::vector<int> parent(size_t(n_nodes) + 1);
  std::iota(parent.begin(), parent.end(), 0);
  auto find = [&](int x) {
    while (parent[size_t(x)] != x) x = parent[size_t(x)] = parent[size_t(parent[size_t(x)])];
    return x;
  };
  auto unite = [&](int a, int b) {
    a = find(a);
    b = find(b);
    if (a != b) parent[size_t(std::max(a, b))] = std::min(a, b);
  };
  std::vector<int> size(size_t(n_nodes) + 1, 0);
  for (const auto& line : lines) {
    int head = -1;            // first projector node of the current stretch
    bool first = true;        // stretch before the first non-diagonal gate
    for (const ProjEvent& ev : line) {
      if (ev.edge < 0) {
        head = -1;
        first = false;
        continue;
      }
      if (ev.edge >= E || cut_of[size_t(ev.edge)] < 0) continue;
      const int node = node_off[size_t(cut_of[size_t(ev.edge)])] + ev.bit;
      if (first) unite(node, zero_node);
      if (head < 0)
        head = node;
      else
        unite(node, head);
    }
  }
  for (int v = 0; v <= n_nodes; ++v) ++size[size_t(find(v))];
  // groups: classes of two or more nodes, or tied to the constant 0
  const int zroot = find(zero_node);
  std::vector<int> group_of(size_t(n_nodes) + 1, -1), class_of(size_t(n_nodes) + 1, -1);
  for (size_t c = 0; c < cuts.size(); ++c) {
    for (int b = 0; b < cut_bits_[c]; ++b) {
      const int v = node_off[c] + b, r = find(v);
      if (r != zroot) {
        if (class_of[size_t(r)] < 0) {
          class_of[size_t(r)] = int(classes_.size());
          classes_.emplace_back();
        }
        classes_[size_t(class_of[size_t(r)])].push_back({int(c), b});
      }
      if (r == zroot || size[size_t(r)] > 1) {
        if (group_of[size_t(r)] < 0) {
          group_of[size_t(r)] = int(groups_.size());
          groups_.emplace_back();
          groups_.back().zero = r == zroot;
        }
        groups_[size_t(group_of[size_t(r)])].bits.push_back({int(c), b});
      }
    }
  }
}

bool SliceZeros::zero(const std::vector<int64_t>& vals) const {
  for (const Group& g : groups_) {
    const int64_t b0 = (vals[size_t(g.bits[0].first)] >> g.bits[0].second) & 1;
    if (g.zero && b0) return true;
    for (const auto& [c, b] : g.bits)
      if (((vals[size_t(c)] >> b) & 1) != b0) return true;
  }
  return false;
}

double SliceZeros::n_nonzero() const { return std::ldexp(1.0, int(classes_.size())); }

bool SliceZeros::list(std::vector<int64_t>* ids, int64_t cap) const {
  if (classes_.size() > 62 || n_nonzero() > double(cap)) return false;
  const int64_t count = int64_t(1) << classes_.size();
  std::vector<int64_t> out(static_cast<size_t>(count));
  std::vector<int64_t> vals(cut_bits_.size());
  for (int64_t a = 0; a < count; ++a) {
    std::fill(vals.begin(), vals.end(), 0);
    for (size_t k = 0; k < classes_.size(); ++k)
      if ((a >> k) & 1)
        for (const auto& [c, b] : classes_[k]) vals[size_t(c)] |= int64_t(1) << b;
    int64_t s = 0;   // mixed radix, first cut most significant
    for (size_t c = 0; c < vals.size(); ++c) s = (s << cut_bits_[c]) | vals[c];
    out[size_t(a)] = s;
  }
  std::sort(out.begin(), out.end());
  *ids = std::move(out);
  return true;
}

}  // namespace qflex
