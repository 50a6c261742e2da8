"""Seeded problem descriptions: circuit + cuts + open tile + contraction order.

A problem is what the C-ABI's planner takes (circuit, cut edges, open tile,
ordering); here it is plain data.  Orderings are lists of (dst, src) tensor-id
pairs: step i contracts tensor `src` into tensor `dst` (the result keeps the id
`dst`); tensor q starts as qubit q's grid tensor.

The rectangular-grid scheme follows the paper's SI A ("Contraction of RQCs on
rectangular grids"): two cuts split an I x J grid into regions A (top-left),
B (top-right), C (bottom-left) and D (bottom-right); A is path independent,
B and the partial region pD are rebuilt per right-cut value, AB = A.B is
reused over the bottom-cut loop, D = pD + its left column per path,
ABD = AB.D, and region C (whose last rows form the open tile) is absorbed
qubit by qubit for the fast-sampling batch.  The figure with the exact region
shapes is not available; the reading used here (A = rows < r0, cols < c0;
right cut on the B-D edge in the last column; bottom cut on the C-D edge in
the last row) gives every region exactly 6 open bonds on a 7x7 grid with
r0 = c0 = 3, matching the 2^(6K) region size the paper states.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

from .circuits import (Circuit, Lattice, diamond_lattice, grid_lattice,
                       random_bitstrings, random_circuit)


@dataclass
class Problem:
    circuit: Circuit
    cut_edges: List[int] = field(default_factory=list)   # indices into circuit.edges
    open_tile: List[int] = field(default_factory=list)   # qubit ids, amplitude-index order
    ordering: Optional[List[Tuple[int, int]]] = None     # (dst, src) pairs
    name: str = ""

    @property
    def n(self) -> int:
        return self.circuit.n


def grid_region_ordering(lat: Lattice, rows: int, cols: int, r0: int, c0: int
                         ) -> List[Tuple[int, int]]:
    """A/B/pD/AB/D/ABD/C ordering on an I x J grid split at row r0, column c0."""
    q = lat.qid
    steps: List[Tuple[int, int]] = []
    a_id, b_id, d_id = q(0, 0), q(0, cols - 1), q(rows - 1, cols - 1)
    for c in range(0, c0):                       # A: columns left->right, top-down
        for r in range(0, r0):
            if (r, c) != (0, 0):
                steps.append((a_id, q(r, c)))
    for c in range(cols - 1, c0 - 1, -1):        # B: columns right->left, top-down
        for r in range(0, r0):
            if (r, c) != (0, cols - 1):
                steps.append((b_id, q(r, c)))
    for c in range(cols - 1, c0, -1):            # pD: columns right->left, bottom-up
        for r in range(rows - 1, r0 - 1, -1):
            if (r, c) != (rows - 1, cols - 1):
                steps.append((d_id, q(r, c)))
    steps.append((a_id, b_id))                   # AB
    for r in range(rows - 1, r0 - 1, -1):        # D = pD + column c0, bottom-up
        if q(r, c0) != d_id:
            steps.append((d_id, q(r, c0)))
    steps.append((a_id, d_id))                   # ABD
    for r in range(r0, rows):                    # region C, row by row, right->left
        for c in range(c0 - 1, -1, -1):
            steps.append((a_id, q(r, c)))
    return steps


def grid_region_cuts(lat: Lattice, rows: int, cols: int, r0: int, c0: int) -> List[int]:
    """Right cut (B-D edge in the last column) first, then the bottom cut."""
    right = lat.edge_id((r0 - 1, cols - 1), (r0, cols - 1))
    bottom = lat.edge_id((rows - 1, c0 - 1), (rows - 1, c0))
    return [right, bottom]


def grid_problem(rows: int, cols: int, t: int, seed: int, *, r0: Optional[int] = None,
                 c0: Optional[int] = None, cuts: bool = True, tile_rows: int = 2,
                 tile_cols: Optional[int] = None, rotations: bool = False,
                 two_qubit: str = "CZ") -> Problem:
    """Rectangular-grid problem with the region ordering and an open tile.

    The tile is the last `tile_rows` rows x first `tile_cols` columns (inside
    region C), in row-major order; tile_rows = 0 gives single amplitudes.
    """
    lat = grid_lattice(rows, cols)
    r0 = rows // 2 if r0 is None else r0
    c0 = cols // 2 if c0 is None else c0
    tile_cols = c0 if tile_cols is None else tile_cols
    circ = random_circuit(lat, t, seed, rotations=rotations, two_qubit=two_qubit)
    tile = [lat.qid(r, c) for r in range(rows - tile_rows, rows) for c in range(tile_cols)]
    return Problem(circ,
                   cut_edges=grid_region_cuts(lat, rows, cols, r0, c0) if cuts else [],
                   open_tile=tile,
                   ordering=grid_region_ordering(lat, rows, cols, r0, c0),
                   name=f"grid{rows}x{cols}_t{t}_s{seed}" + ("_iswap" if two_qubit == "ISWAP" else ""))


def row_major_ordering(lat: Lattice) -> List[Tuple[int, int]]:
    """Absorb every qubit into qubit 0 in id order (small grids only)."""
    return [(0, q) for q in range(1, lat.n)]


# --------------------------------------------------------------------------
# Named workloads (the shapes follow the paper's runs; the circuits are
# seeded synthetic stand-ins for the published instances, which are not used)
# --------------------------------------------------------------------------

def c1_problem(seed: int = 0, full_tile: bool = False) -> Problem:
    """4x4 grid, depth 1+16+1, no cuts; tile = all 16 qubits when full_tile."""
    lat = grid_lattice(4, 4)
    circ = random_circuit(lat, 16, seed)
    tile = list(range(16)) if full_tile else []
    return Problem(circ, [], tile, grid_region_ordering(lat, 4, 4, 2, 2),
                   name=f"c1_4x4_t16_s{seed}")


def c2_problem(seed: int = 0, t: int = 32, two_qubit: str = "CZ") -> Problem:
    """7x7 grid, depth 1+t+1, 2 cuts, 6-qubit open tile (rows 5-6, cols 0-2).

    With two_qubit="ISWAP" every bond carries 2 bits per gate, so depth
    1+t/2+1 with iSWAPs has the bond dimensions of depth 1+t+1 with CZs
    (Methods, "Overview of the simulator": Schmidt rank 4 vs 2)."""
    p = grid_problem(7, 7, t, seed, r0=3, c0=3, cuts=True, tile_rows=2, tile_cols=3,
                     two_qubit=two_qubit)
    p.name = f"grid7x7_t{t}_s{seed}" + ("_iswap" if two_qubit == "ISWAP" else "")
    return p


def c4_problem(seed: int = 0) -> Problem:
    """7x7 grid, depth 1+40+1 (bond dimension 32), same structure as c2."""
    return c2_problem(seed, t=40)


def workload_bitstrings(problem: Problem, count: int, seed: int) -> np.ndarray:
    return random_bitstrings(problem.n, count, seed)


def rotation_batch(count: int = 256, seed: int = 0) -> List[Problem]:
    """Batch of uneven rotation circuits: grids I, J ~ U{4, 5, 6}, depth
    1+t+1 with t ~ U{16..32}, every non-CZ gate R_P(theta) with P uniform in
    {X, Y, Z} and theta ~ U[0, 2 pi), no cuts, one amplitude per circuit
    (region ordering split at the middle row and column)."""
    rng = np.random.default_rng([seed, 0xC5])
    out = []
    for i in range(count):
        rows, cols = int(rng.integers(4, 7)), int(rng.integers(4, 7))
        t = int(rng.integers(16, 33))
        p = grid_problem(rows, cols, t, seed * 100003 + i, cuts=False, tile_rows=0,
                         rotations=True)
        p.name = f"rot{rows}x{cols}_t{t}_{i}"
        out.append(p)
    return out


def diamond_problem(t: int, seed: int, size: int = 12, n_cuts: int = 4, c_split=None,
                    c_rows: int = 2) -> Problem:
    """Bristlecone-like diamond without its two degree-1 corners (size 12:
    70 qubits, rows of 3,5,7,9,11,11,9,7,5,3 qubits).

    The figure with the paper's regions is not available; this reading keeps
    the structure the text gives (Methods "Cutting indexes": four cuts of
    2^4, regions A and B contracted per path, A.B then the path-independent
    region C holding the open tile):
      A = columns <= c_split of the upper rows, B = the rest of the upper rows,
      C = the last c_rows rows (the open tile, 2^|C| amplitudes);
      cuts = the A-B bonds of the first n_cuts rows.
    Orders: A row by row, left to right; B row by row, left to right down to
    the widest row and right to left below it; AB = A.B; C absorbed row by
    row.  With size 12 every intermediate stays within 7 bonds (2^28
    entries at bond dimension 16), A has rank 6 and B rank 7.
    """
    lat = diamond_lattice(drop_corners=True) if size == 12 else _small_diamond(size)
    rows = sorted({r for r, _ in lat.coords})
    r_first, r_last = rows[0], rows[-1]
    widths = {r: sum(1 for rr, _ in lat.coords if rr == r) for r in rows}
    r_wide = max(rows, key=lambda r: (widths[r], -r))
    cs = sorted({c for _, c in lat.coords})
    c_split = (cs[0] + cs[-1]) // 2 - 1 if c_split is None else c_split
    circ = random_circuit(lat, t, seed)
    upper = [r for r in rows if r <= r_last - c_rows]
    in_row = lambda r: sorted(c for rr, c in lat.coords if rr == r)
    A = [(r, c) for r in upper for c in in_row(r) if c <= c_split]
    B = []
    for r in upper:
        cols = [c for c in in_row(r) if c > c_split]
        B += [(r, c) for c in (cols if r <= r_wide else cols[::-1])]
    C = [(r, c) for r in rows if r > r_last - c_rows for c in in_row(r)]
    q = lat.qid
    steps: List[Tuple[int, int]] = []
    a_id, b_id = q(*A[0]), q(*B[0])
    steps += [(a_id, q(*x)) for x in A[1:]]
    steps += [(b_id, q(*x)) for x in B[1:]]
    steps.append((a_id, b_id))
    steps += [(a_id, q(*x)) for x in C]
    cut_rows = [r for r in upper if any(c == c_split for c in in_row(r))
                and any(c == c_split + 1 for c in in_row(r))][:n_cuts]
    cuts = [lat.edge_id((r, c_split), (r, c_split + 1)) for r in cut_rows]
    tile = [q(*x) for x in C]
    return Problem(circ, cuts, tile, steps, name=f"{lat.name}_t{t}_s{seed}")


def _small_diamond(size: int) -> Lattice:
    """Diamond of a size x size rotated lattice (size even), corners dropped."""
    pts = []
    for x in range(size):
        for y in range(size):
            if (x + y) % 2 == 0 and (x, y) not in ((0, 0), (size - 1, size - 1)):
                pts.append(((x + y) // 2, (x - y) // 2 + size // 2 - 1))
    return Lattice(pts, name=f"diamond{size}_{len(pts)}")
