"""Brute-force FP64 state-vector amplitudes (oracle; test infrastructure only).

amp(x) = <x| U |0^n>, with U the product of the circuit's gates in cycle order
(Methods, "Overview of the simulator": the network's contraction with input
and output deltas gives exactly this amplitude).  This is the plain definition
the contraction must reach, used for n <= ~20 qubits.

The state is a complex128 array of shape (2,)*n; axis q is qubit q, so qubit 0
is the most significant bit of the flat state index.

Slice variants (Methods, "Cutting indexes"): cutting the bond of edge e fixes
its multi-index to a value v; under the CZ split reading (lower-index qubit
carries |k><k|, the other Z^k; bond multi-index sum_m k_m 2^{K_e-1-m} with the
edge's CZs in time order, first most significant), the slice equals the same
circuit with every CZ on e replaced by the non-unitary |k_m><k_m| (x) Z^{k_m}.
An iSWAP takes 2 bits k of the bond value (high bit first) and is replaced by
A_k (x) B_k of its Pauli split (gates.iswap_half).
"""
from __future__ import annotations

from typing import Dict, Optional, Sequence

import numpy as np

from . import gates as G


def _apply_1q(psi: np.ndarray, U: np.ndarray, q: int) -> np.ndarray:
    out = np.tensordot(U, psi, axes=([1], [q]))
    return np.moveaxis(out, 0, q)


def _apply_diag2(psi: np.ndarray, da: np.ndarray, a: int, db: np.ndarray, b: int) -> np.ndarray:
    shape = [1] * psi.ndim
    shape[a] = 2
    psi = psi * da.reshape(shape)
    shape = [1] * psi.ndim
    shape[b] = 2
    return psi * db.reshape(shape)


def _apply_2q(psi: np.ndarray, U: np.ndarray, a: int, b: int) -> np.ndarray:
    """Apply a 4x4 matrix on qubits (a, b), a the first (most significant) factor."""
    out = np.tensordot(U.reshape(2, 2, 2, 2), psi, axes=([2, 3], [a, b]))
    return np.moveaxis(out, (0, 1), (a, b))


def gate_bits(kind: str) -> int:
    """Bond bits one two-qubit gate adds to its edge (Schmidt rank 2 or 4)."""
    return {"CZ": 1, "ISWAP": 2}.get(kind, 0)


def _cz(psi: np.ndarray, a: int, b: int) -> np.ndarray:
    psi = psi.copy()
    idx = [slice(None)] * psi.ndim
    idx[a] = 1
    idx[b] = 1
    psi[tuple(idx)] *= -1.0
    return psi


def final_state(circ, angles: Optional[np.ndarray] = None,
                cut_values: Optional[Dict[int, int]] = None) -> np.ndarray:
    """U|0^n> as a (2,)*n array; `cut_values` maps edge index -> fixed bond value."""
    n = circ.n
    angles = circ.angles if angles is None else np.asarray(angles, dtype=np.float64)
    cut_values = cut_values or {}
    K = {}
    for g in circ.gates:
        if gate_bits(g.kind):
            e = circ.lattice.edge_index[(min(g.q0, g.q1), max(g.q0, g.q1))]
            K[e] = K.get(e, 0) + gate_bits(g.kind)
    seen: Dict[int, int] = {}
    psi = np.zeros((2,) * n, dtype=np.complex128)
    psi[(0,) * n] = 1.0
    for g in sorted(circ.gates, key=lambda g: g.cycle):
        w = gate_bits(g.kind)
        if w:
            a, b = min(g.q0, g.q1), max(g.q0, g.q1)
            e = circ.lattice.edge_index[(a, b)]
            used = seen.get(e, 0)
            if e in cut_values:
                k = (cut_values[e] >> (K[e] - used - w)) & ((1 << w) - 1)
                if g.kind == "CZ":
                    psi = _apply_diag2(psi, np.diag(G.cz_half("proj", k)), a,
                                       np.diag(G.cz_half("z", k)), b)
                else:
                    psi = _apply_1q(_apply_1q(psi, G.iswap_half("a", k), a), G.iswap_half("b", k), b)
            elif g.kind == "CZ":
                psi = _cz(psi, a, b)
            else:
                psi = _apply_2q(psi, G.ISWAP, a, b)
            seen[e] = used + w
        else:
            psi = _apply_1q(psi, G.single_qubit_matrix(g.kind, angles, g.param), g.q0)
    return psi


def tile_amplitudes_from_state(psi: np.ndarray, bitstring: Sequence[int],
                               tile: Sequence[int]) -> np.ndarray:
    """Amplitudes for `bitstring` with the tile qubits' bits enumerated.

    Tile index j = sum_t b_{tile[t]} 2^{|tile|-1-t} (first tile qubit most
    significant); the bitstring's own bits on tile qubits are ignored.
    """
    n = psi.ndim
    nt = len(tile)
    out = np.empty(1 << nt, dtype=np.complex128)
    x = [int(b) for b in bitstring]
    for j in range(1 << nt):
        for t, q in enumerate(tile):
            x[q] = (j >> (nt - 1 - t)) & 1
        out[j] = psi[tuple(x)]
    return out


def amplitudes(circ, bitstrings: np.ndarray, tile: Sequence[int] = (),
               angles: Optional[np.ndarray] = None,
               cut_values: Optional[Dict[int, int]] = None) -> np.ndarray:
    """complex128 [n_bs, 2^|tile|] amplitudes by state-vector simulation."""
    psi = final_state(circ, angles, cut_values)
    bitstrings = np.atleast_2d(bitstrings)
    return np.stack([tile_amplitudes_from_state(psi, b, tile) for b in bitstrings])
