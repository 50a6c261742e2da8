"""Seeded synthetic random quantum circuits (RQCs) on square-grid subsets.

This module only *places* gates: it yields gate names, the qubits they act on,
their cycle and, for rotation gates, an index into an angle vector.  It holds
none of the simulation arithmetic (no gate matrices, no contraction); the
oracle and the CUDA path each turn these names into numbers on their own.

Circuit rules follow the paper's Methods, "Revised set of Random Quantum
Circuits", rules (1)-(5):
  (1) a first layer of H on every qubit (cycle 0);
  (2) then t cycles of CZ layers, cycling through 8 layer patterns;
  (3) in a CZ cycle, an idle qubit that had a CZ in the previous cycle gets
      X^1/2 or Y^1/2 with equal probability;
  (4) an idle qubit whose previous-cycle gate was X^1/2, Y^1/2 or H gets T;
  (5) a final layer of H on every qubit (cycle t+1).
Depth "1+t+1" therefore means t CZ cycles.

The 8 CZ layer patterns appear only in a figure (Fig. "coverings"), so this
module fixes a reading that satisfies every textual constraint of the paper
(Methods, "Overview of the simulator": each qubit shares exactly one CZ with
each neighbour per 8 cycles; Methods, "Revised set": no two consecutive
horizontal or vertical layers):
  H(a, b): edges (r, c)-(r, c+1) with c = a (mod 2), r = b (mod 2)
  V(a, b): edges (r, c)-(r+1, c) with r = a (mod 2), c = b (mod 2)
  cycle order H00, V00, H11, V11, H01, V01, H10, V10, repeating.

The rotation variant replaces every non-CZ gate (including the H and T slots)
by R_P(theta), P uniform in {X, Y, Z}, theta uniform in [0, 2 pi).

The iSWAP variant (Methods, "Revised set of RQCs": replacing the CZs by
iSWAPs makes the circuits harder) places an ISWAP wherever the CZ variant
places a CZ, with the same layer patterns and the same single-qubit rules
(rule (3) keyed on "a two-qubit gate in the previous cycle"); for the same
seed the two variants share every placement draw.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Gate kind names; the integer codes are the C-ABI's gate kinds.
KINDS = ("H", "T", "SX", "SY", "CZ", "RX", "RY", "RZ", "ISWAP")
TWO_QUBIT = ("CZ", "ISWAP")
KIND_ID = {k: i for i, k in enumerate(KINDS)}

_LAYER_ORDER = (("H", 0, 0), ("V", 0, 0), ("H", 1, 1), ("V", 1, 1),
                ("H", 0, 1), ("V", 0, 1), ("H", 1, 0), ("V", 1, 0))


@dataclass
class Lattice:
    """Qubits at square-grid coordinates; edges join grid neighbours.

    Qubit ids are assigned in row-major order of (r, c).  Edges are (p, q)
    pairs with p < q, sorted.
    """
    coords: List[Tuple[int, int]]
    name: str = ""
    edges: List[Tuple[int, int]] = field(default_factory=list)

    def __post_init__(self):
        self.coords = sorted(self.coords)
        self.index = {rc: i for i, rc in enumerate(self.coords)}
        if not self.edges:
            e = []
            for i, (r, c) in enumerate(self.coords):
                for nb in ((r, c + 1), (r + 1, c)):
                    j = self.index.get(nb)
                    if j is not None:
                        e.append((min(i, j), max(i, j)))
            self.edges = sorted(e)
        self.edge_index = {e: k for k, e in enumerate(self.edges)}

    @property
    def n(self) -> int:
        return len(self.coords)

    def qid(self, r: int, c: int) -> int:
        return self.index[(r, c)]

    def edge_id(self, a: Tuple[int, int], b: Tuple[int, int]) -> int:
        p, q = self.qid(*a), self.qid(*b)
        return self.edge_index[(min(p, q), max(p, q))]

    def neighbours(self, q: int) -> List[int]:
        out = [b if a == q else a for (a, b) in self.edges if q in (a, b)]
        return sorted(out)


def grid_lattice(rows: int, cols: int) -> Lattice:
    """I x J square grid, qubit id = r * J + c."""
    return Lattice([(r, c) for r in range(rows) for c in range(cols)],
                   name=f"grid{rows}x{cols}")


def diamond_lattice(drop_corners: bool = False) -> Lattice:
    """Bristlecone-like 72-qubit diamond on a 45-degree rotated square lattice.

    Rotated-lattice sites (x, y), 0 <= x, y <= 11, x + y even (72 sites),
    neighbours (x +- 1, y +- 1).  Grid coordinates r = (x + y) / 2,
    c = (x - y) / 2 + 5 map rotated-lattice neighbours to grid neighbours.
    The two corners (0, 0) and (11, 11) are the only degree-1 qubits; dropping
    them leaves 70 qubits inside a 10 x 11 box (Methods, "Contraction of the
    3D tensor network"; Methods, "Simulation of Bristlecone compared to
    rectangular grids").  Device coordinates are a reading of a figure that is
    not available, so they are not pinned to the hardware layout.
    """
    pts = []
    for x in range(12):
        for y in range(12):
            if (x + y) % 2 == 0:
                if drop_corners and (x, y) in ((0, 0), (11, 11)):
                    continue
                pts.append(((x + y) // 2, (x - y) // 2 + 5))
    return Lattice(pts, name="bris70" if drop_corners else "bris72")


def layer_edges(lat: Lattice, layer: int) -> List[Tuple[int, int]]:
    """Edges of CZ layer pattern `layer` (0..7, taken mod 8) present in `lat`."""
    kind, a, b = _LAYER_ORDER[layer % 8]
    out = []
    for (p, q) in lat.edges:
        (r0, c0), (r1, c1) = lat.coords[p], lat.coords[q]
        if kind == "H" and r0 == r1:
            if min(c0, c1) % 2 == a and r0 % 2 == b:
                out.append((p, q))
        elif kind == "V" and c0 == c1:
            if min(r0, r1) % 2 == a and c0 % 2 == b:
                out.append((p, q))
    return out


@dataclass
class Gate:
    cycle: int
    kind: str
    q0: int
    q1: int = -1
    param: int = -1  # index into Circuit.angles for RX/RY/RZ, else -1


@dataclass
class Circuit:
    lattice: Lattice
    depth: int                    # t, the number of CZ cycles
    gates: List[Gate]
    angles: np.ndarray            # float64 [n_params]
    seed: int = 0

    @property
    def n(self) -> int:
        return self.lattice.n

    @property
    def edges(self):
        return self.lattice.edges

    @property
    def n_params(self) -> int:
        return int(self.angles.shape[0])

    def gate_array(self) -> np.ndarray:
        """Gates as an int32 [n_gates, 5] array: cycle, kind, q0, q1, param."""
        return np.array([[g.cycle, KIND_ID[g.kind], g.q0, g.q1, g.param]
                         for g in self.gates], dtype=np.int32).reshape(-1, 5)

    def edge_array(self) -> np.ndarray:
        return np.array(self.lattice.edges, dtype=np.int32).reshape(-1, 2)

    def with_angles(self, angles: np.ndarray) -> "Circuit":
        return Circuit(self.lattice, self.depth, self.gates,
                       np.asarray(angles, dtype=np.float64).copy(), self.seed)


def random_circuit(lat: Lattice, t: int, seed: int, rotations: bool = False,
                   two_qubit: str = "CZ") -> Circuit:
    """Seeded RQC of depth 1+t+1 on `lat` (rules (1)-(5) above).

    Layout draws and rotation draws come from separate streams, so the
    rotation variant keeps the gate placement of the plain circuit.
    `two_qubit` is "CZ" or "ISWAP" (the gate placed on every active edge).
    """
    if two_qubit not in TWO_QUBIT:
        raise ValueError(f"two_qubit must be one of {TWO_QUBIT}")
    rng = np.random.default_rng([seed, 0x51F1])
    rrng = np.random.default_rng([seed, 0x52A7])
    n = lat.n
    gates: List[Gate] = [Gate(0, "H", q) for q in range(n)]
    prev: List[Optional[str]] = ["H"] * n
    for k in range(1, t + 1):
        active = layer_edges(lat, k - 1)
        busy = set()
        for (p, q) in active:
            busy.add(p)
            busy.add(q)
        cur: List[Optional[str]] = [None] * n
        for q in range(n):
            if q in busy:
                cur[q] = two_qubit
                continue
            g = None
            if prev[q] == two_qubit:
                g = "SX" if int(rng.integers(2)) == 0 else "SY"
            elif prev[q] in ("SX", "SY", "H"):
                g = "T"
            if g is not None:
                gates.append(Gate(k, g, q))
                cur[q] = g
        for (p, q) in active:
            gates.append(Gate(k, two_qubit, p, q))
        prev = cur
    gates.extend(Gate(t + 1, "H", q) for q in range(n))
    angles: List[float] = []
    if rotations:
        for g in gates:
            if g.kind not in TWO_QUBIT:
                g.kind = ("RX", "RY", "RZ")[int(rrng.integers(3))]
                g.param = len(angles)
                angles.append(float(rrng.uniform(0.0, 2.0 * np.pi)))
    return Circuit(lat, t, gates, np.array(angles, dtype=np.float64), seed)


def random_bitstrings(n_qubits: int, count: int, seed: int) -> np.ndarray:
    """uint8 [count, n_qubits] uniform random output bits (index = qubit id)."""
    rng = np.random.default_rng([seed, 0xB175])
    return rng.integers(0, 2, size=(count, n_qubits), dtype=np.uint8)


def two_qubit_counts(circ: Circuit) -> np.ndarray:
    """Number of two-qubit gates (CZ or ISWAP) on each lattice edge."""
    cnt = np.zeros(len(circ.edges), dtype=np.int64)
    idx = circ.lattice.edge_index
    for g in circ.gates:
        if g.kind in TWO_QUBIT:
            cnt[idx[(min(g.q0, g.q1), max(g.q0, g.q1))]] += 1
    return cnt


def cz_counts(circ: Circuit) -> np.ndarray:
    """Number of CZ gates on each lattice edge (the bond exponent K_e)."""
    cnt = np.zeros(len(circ.edges), dtype=np.int64)
    idx = circ.lattice.edge_index
    for g in circ.gates:
        if g.kind == "CZ":
            cnt[idx[(min(g.q0, g.q1), max(g.q0, g.q1))]] += 1
    return cnt
