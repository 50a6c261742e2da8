// Paths that vanish identically (host code, slices.cpp).
//
// A path fixes the values of the cut bonds (Methods, "Cutting indexes").  On
// one qubit, the CZ projector halves |k><k| (carried by the lower-index
// qubit of each CZ) multiply through diagonal gates (T, R_Z, the Z halves of
// other CZs): |j><j| D |k><k| = 0 unless j = k.  A projector met before the
// qubit's first non-diagonal gate acts on the input |0> and needs k = 0.  So
// a path whose cut values give two different bits inside one diagonal
// stretch, or a 1 inside a first stretch, contributes exactly zero for every
// bitstring and every angle.
#pragma once

#include <cstdint>
#include <utility>
#include <vector>

namespace qflex {

// One qubit's time line reduced to what the rule needs: a CZ projector half
// on `edge`, bit `bit` of that edge's value (edge >= 0), or a non-diagonal
// gate closing the stretch (edge = -1).  Diagonal gates are left out.
struct ProjEvent {
  int edge;
  int bit;
};
using ProjLines = std::vector<std::vector<ProjEvent>>;   // per qubit, time order

class SliceZeros {
 public:
  SliceZeros() = default;
  // edge_bits: K_e per edge; cuts: edge ids, first most significant.
  SliceZeros(const ProjLines& lines, const std::vector<int>& edge_bits, const std::vector<int>& cuts);

  bool any() const { return !groups_.empty(); }
  // vals: the path's value per cut
  bool zero(const std::vector<int64_t>& vals) const;
  // paths not ruled out: 2^(bit classes not tied to 0)
  double n_nonzero() const;
  // their ids, ascending; false (ids untouched) when there are more than cap
  bool list(std::vector<int64_t>* ids, int64_t cap) const;

 private:
  struct Group {
    std::vector<std::pair<int, int>> bits;   // (cut, bit) that must agree
    bool zero = false;                       // ... and be 0
  };
  std::vector<Group> groups_;
  std::vector<std::vector<std::pair<int, int>>> classes_;   // free classes (cut, bit)
  std::vector<int> cut_bits_;
};

}  // namespace qflex
