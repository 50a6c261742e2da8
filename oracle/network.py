"""FP64 tensor-network contraction of an RQC (oracle; test infrastructure only).

Follows the paper's construction step by step, in plain NumPy:

* Grid tensors (Methods, "Overview of the simulator" and "Contraction of the
  3D tensor network"): every gate on qubit q, in time order, is contracted
  into one tensor T_q[o, e_1, ..., e_d].  One-qubit gates are rank-2 tensors;
  each CZ contributes one binary bond index through its rank-2 Schmidt split
  (-1)^{ab} = sum_k d_{a,k} (-1)^{k b} (lower-index qubit: |k><k|, the other:
  Z^k); each iSWAP contributes two bits through its rank-4 split
  iSWAP = sum_k A_k (x) B_k (gates.iswap_half).  The bits of one edge, in
  time order with the first most significant, form that edge's bond of
  dimension 2^{K_e}; bonds are ordered by neighbour id; o is the output leg
  (input |0>).
* Cuts (Methods, "Cutting indexes"): fixing the value of every cut bond gives
  a "path"; the amplitude is the sum over all paths.  Slice id s is decoded in
  mixed radix 2^{K_e} over the cut list, first cut most significant.
* Pairwise contraction along a given ordering of (dst, src) pairs, each a
  tensordot over the shared bonds (any order gives the same exact value).
* Open tile (Methods, "Fast sampling technique"): output legs of tile qubits
  stay open, so one contraction gives 2^{|tile|} amplitudes.
* Fraction-f sums (Methods, "Summing a fraction of the paths"): summing a
  subset of slices, with no rescaling.
* Paths that vanish identically (projector_runs): CZ projector halves on
  one qubit with only diagonal gates between them must agree.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import gates as G


_GATE_BITS = {"CZ": 1, "ISWAP": 2}


def bond_exponents(circ) -> np.ndarray:
    """K_e: bond bits of each edge, 1 per CZ and 2 per iSWAP (bond dimension 2^{K_e})."""
    K = np.zeros(len(circ.edges), dtype=np.int64)
    for g in circ.gates:
        if g.kind in _GATE_BITS:
            K[circ.lattice.edge_index[(min(g.q0, g.q1), max(g.q0, g.q1))]] += _GATE_BITS[g.kind]
    return K


def grid_tensor(circ, q: int, angles: Optional[np.ndarray] = None
                ) -> Tuple[np.ndarray, List[tuple]]:
    """T_q with legs [('o', q)] + [('e', edge) for neighbours in ascending id]."""
    angles = circ.angles if angles is None else np.asarray(angles, dtype=np.float64)
    lat = circ.lattice
    t = np.array([1.0, 0.0], dtype=np.complex128)      # |0>, axis 0 = qubit state
    bit_edges: List[int] = []                           # edge of each bond bit, time order
    for g in sorted((g for g in circ.gates if q in (g.q0, g.q1)), key=lambda g: g.cycle):
        if g.kind == "CZ":
            other = g.q1 if g.q0 == q else g.q0
            role = "proj" if q < other else "z"
            d0 = np.diag(G.cz_half(role, 0))
            d1 = np.diag(G.cz_half(role, 1))
            shp = (2,) + (1,) * (t.ndim - 1)
            t = np.stack([d0.reshape(shp) * t, d1.reshape(shp) * t], axis=-1)
            bit_edges.append(lat.edge_index[(min(q, other), max(q, other))])
        elif g.kind == "ISWAP":
            other = g.q1 if g.q0 == q else g.q0
            role = "a" if q < other else "b"
            terms = [np.tensordot(G.iswap_half(role, k), t, axes=([1], [0])) for k in range(4)]
            t = np.stack(terms, axis=-1).reshape(t.shape + (2, 2))   # k = 2 hi + lo, hi first
            e = lat.edge_index[(min(q, other), max(q, other))]
            bit_edges.extend([e, e])
        else:
            U = G.single_qubit_matrix(g.kind, angles, g.param)
            t = np.tensordot(U, t, axes=([1], [0]))
    nbrs = lat.neighbours(q)
    legs = [("o", q)]
    axes = [0]
    dims = [2]
    for p in nbrs:
        e = lat.edge_index[(min(p, q), max(p, q))]
        pos = [1 + i for i, be in enumerate(bit_edges) if be == e]
        axes.extend(pos)
        dims.append(1 << len(pos))
        legs.append(("e", e))
    t = np.transpose(t, axes).reshape(dims)
    return t, legs


def all_grid_tensors(circ, angles=None):
    return [grid_tensor(circ, q, angles) for q in range(circ.n)]


def n_slices(circ, cut_edges: Sequence[int]) -> int:
    K = bond_exponents(circ)
    P = 1
    for e in cut_edges:
        P *= 1 << int(K[e])
    return P


def slice_values(circ, cut_edges: Sequence[int], s: int) -> Dict[int, int]:
    """Decode slice id s into cut-bond values (mixed radix, first cut most significant)."""
    K = bond_exponents(circ)
    vals = {}
    for e in reversed(list(cut_edges)):
        r = 1 << int(K[e])
        vals[e] = s % r
        s //= r
    return vals


# Gates whose matrix is diagonal for every angle (the Z half of a CZ and its
# projector half are diagonal too; iSWAP halves are not).
_DIAGONAL_1Q = ("T", "RZ")


def projector_runs(circ, cut_edges: Sequence[int]) -> Tuple[List[List[Tuple[int, int]]], List[bool]]:
    """Per qubit, the maximal stretches of its time line free of non-diagonal
    gates, each reduced to the CZ projector halves |k><k| it holds on cut
    edges, as (edge, bit position in the edge's value) pairs; and whether
    the stretch is the first one (it then acts on the input |0>).

    Projectors multiply through diagonal gates: |j><j| D |k><k| = 0 unless
    j = k, and |k><k| |0> = 0 unless k = 0.  So a path whose cut values give
    two different bits inside one stretch, or a 1 inside a first stretch, is
    zero for every bitstring and every angle (Methods, "Cutting indexes": a
    path is the network with the cut bonds fixed)."""
    K = bond_exponents(circ)
    cut = set(int(e) for e in cut_edges)
    runs: List[List[Tuple[int, int]]] = []
    first: List[bool] = []
    for q in range(circ.n):
        used: Dict[int, int] = {}
        cur: List[Tuple[int, int]] = []
        is_first = True
        for g in sorted((g for g in circ.gates if q in (g.q0, g.q1)), key=lambda g: g.cycle):
            if g.kind in ("CZ", "ISWAP"):
                e = circ.lattice.edge_index[(min(g.q0, g.q1), max(g.q0, g.q1))]
                j = used.get(e, 0)
                used[e] = j + _GATE_BITS[g.kind]
                if g.kind == "CZ":
                    other = g.q1 if g.q0 == q else g.q0
                    if q < other and e in cut:
                        cur.append((e, int(K[e]) - 1 - j))   # first bit in time = most significant
                    continue
            elif g.kind in _DIAGONAL_1Q:
                continue
            # a non-diagonal gate closes the stretch
            runs.append(cur)
            first.append(is_first)
            cur, is_first = [], False
        runs.append(cur)
        first.append(is_first)
    return runs, first


def _zero_by_runs(runs, first, vals: Dict[int, int]) -> bool:
    for members, is_first in zip(runs, first):
        bits = {(vals[e] >> b) & 1 for e, b in members}
        if len(bits) > 1 or (is_first and 1 in bits):
            return True
    return False


def structurally_zero(circ, cut_edges: Sequence[int], s: int) -> bool:
    """Whether path s vanishes identically by the projector rule of
    projector_runs.  (The bitstring's <x_q| after a qubit's last stretch
    would fix that stretch's bits too; it is left out, so the rule holds for
    every bitstring.)"""
    return _zero_by_runs(*projector_runs(circ, cut_edges), slice_values(circ, cut_edges, s))


def nonzero_slices(circ, cut_edges: Sequence[int]) -> List[int]:
    """Ascending ids of the paths that projector_runs does not rule out."""
    runs, first = projector_runs(circ, cut_edges)
    K = bond_exponents(circ)
    out = []
    for s in range(n_slices(circ, cut_edges)):
        vals, rest = {}, s                       # mixed radix, as slice_values
        for e in reversed(list(cut_edges)):
            vals[e] = rest % (1 << int(K[e]))
            rest //= 1 << int(K[e])
        if not _zero_by_runs(runs, first, vals):
            out.append(s)
    return out


def _fix(arr: np.ndarray, legs: List[tuple], fixed: Dict[tuple, int]):
    for leg, v in fixed.items():
        if leg in legs:
            ax = legs.index(leg)
            arr = np.take(arr, v, axis=ax)
            legs = legs[:ax] + legs[ax + 1:]
    return arr, legs


def contract_pair(a, la, b, lb):
    shared = [l for l in la if l in lb]
    ia = [la.index(l) for l in shared]
    ib = [lb.index(l) for l in shared]
    out = np.tensordot(a, b, axes=(ia, ib))
    return out, [l for l in la if l not in shared] + [l for l in lb if l not in shared]


def slice_amplitudes(problem, bitstring: Sequence[int], s: int,
                     angles: Optional[np.ndarray] = None, tensors=None) -> np.ndarray:
    """Contribution of slice (path) s to the tile amplitudes of `bitstring`."""
    circ = problem.circuit
    tensors = all_grid_tensors(circ, angles) if tensors is None else tensors
    tile = list(problem.open_tile)
    vals = slice_values(circ, problem.cut_edges, s)
    fixed_bonds = {("e", e): v for e, v in vals.items()}
    net = {}
    for q, (arr, legs) in enumerate(tensors):
        fx = dict(fixed_bonds)
        if q not in tile:
            fx[("o", q)] = int(bitstring[q])
        net[q] = _fix(arr, legs, fx)
    order = problem.ordering or [(0, q) for q in range(1, circ.n)]
    for dst, src in order:
        a, la = net.pop(dst)
        b, lb = net.pop(src)
        net[dst] = contract_pair(a, la, b, lb)
    assert len(net) == 1, "ordering must contract every tensor into one"
    (arr, legs), = net.values()
    want = [("o", q) for q in tile]
    assert sorted(legs) == sorted(want), f"open legs {legs} != tile {want}"
    arr = np.transpose(arr, [legs.index(l) for l in want]) if want else arr
    return np.asarray(arr, dtype=np.complex128).reshape(-1)


def amplitudes(problem, bitstrings: np.ndarray, slices: Optional[Sequence[int]] = None,
               angles: Optional[np.ndarray] = None) -> np.ndarray:
    """complex128 [n_bs, 2^|tile|]: sum over `slices` (all slices when None),
    accumulated in ascending slice order."""
    circ = problem.circuit
    tensors = all_grid_tensors(circ, angles)
    P = n_slices(circ, problem.cut_edges)
    sl = range(P) if slices is None else sorted(int(s) for s in slices)
    bitstrings = np.atleast_2d(bitstrings)
    out = np.zeros((len(bitstrings), 1 << len(problem.open_tile)), dtype=np.complex128)
    for i, b in enumerate(bitstrings):
        for s in sl:
            out[i] += slice_amplitudes(problem, b, s, angles, tensors)
    return out
