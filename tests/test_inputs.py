"""Invariants of the seeded circuit generator (no GPU)."""
import collections

import numpy as np
import pytest

from qflex_inputs import (c2_problem, cz_counts, diamond_lattice, grid_lattice,
                          grid_problem, layer_edges, random_circuit)


@pytest.mark.parametrize("lat", [grid_lattice(5, 6), diamond_lattice()])
def test_each_edge_once_per_8_cycles(lat):
    seen = collections.Counter()
    for L in range(8):
        busy = collections.Counter()
        for (p, q) in layer_edges(lat, L):
            seen[(p, q)] += 1
            busy[p] += 1
            busy[q] += 1
        assert max(busy.values(), default=0) <= 1        # a layer touches a qubit once
    assert all(seen[e] == 1 for e in lat.edges)


def test_layers_alternate_horizontal_vertical():
    lat = grid_lattice(4, 4)
    kinds = []
    for L in range(16):
        e = layer_edges(lat, L)
        (r0, _), (r1, _) = lat.coords[e[0][0]], lat.coords[e[0][1]]
        kinds.append("H" if r0 == r1 else "V")
    assert all(a != b for a, b in zip(kinds, kinds[1:]))


def test_single_qubit_gate_rules():
    circ = random_circuit(grid_lattice(4, 5), 24, seed=11)
    n = circ.n
    by_cycle = collections.defaultdict(dict)
    for g in circ.gates:
        by_cycle[g.cycle][g.q0] = g.kind
        if g.kind == "CZ":
            by_cycle[g.cycle][g.q1] = "CZ"
    assert all(by_cycle[0][q] == "H" for q in range(n))
    assert all(by_cycle[25][q] == "H" for q in range(n))
    for k in range(1, 25):
        for q in range(n):
            prev = by_cycle[k - 1].get(q)
            cur = by_cycle[k].get(q)
            if cur == "CZ":
                continue
            if prev == "CZ":
                assert cur in ("SX", "SY")
            elif prev in ("SX", "SY", "H"):
                assert cur == "T"
            else:
                assert cur is None
    # T is never placed right after a CZ
    for g in circ.gates:
        if g.kind == "T":
            assert by_cycle[g.cycle - 1].get(g.q0) in ("SX", "SY", "H")


def test_bond_dimension_is_t_over_8():
    for t in (8, 16, 32, 40):
        circ = random_circuit(grid_lattice(3, 4), t, seed=t)
        assert set(cz_counts(circ).tolist()) == {t // 8}


def test_diamond_geometry():
    lat = diamond_lattice()
    assert lat.n == 72
    deg = collections.Counter()
    for a, b in lat.edges:
        deg[a] += 1
        deg[b] += 1
    ones = sorted(lat.coords[q] for q in range(72) if deg[q] == 1)
    assert len(ones) == 2
    lat70 = diamond_lattice(drop_corners=True)
    rs = [r for r, _ in lat70.coords]
    cs = [c for _, c in lat70.coords]
    assert lat70.n == 70 and max(rs) - min(rs) + 1 == 10 and max(cs) - min(cs) + 1 == 11


def test_rotation_variant_keeps_layout():
    a = random_circuit(grid_lattice(3, 3), 16, seed=5)
    b = random_circuit(grid_lattice(3, 3), 16, seed=5, rotations=True)
    assert [(g.cycle, g.q0, g.q1) for g in a.gates] == [(g.cycle, g.q0, g.q1) for g in b.gates]
    assert b.n_params == sum(g.kind != "CZ" for g in a.gates)
    assert all(g.kind in ("RX", "RY", "RZ", "CZ") for g in b.gates)
    assert np.all((b.angles >= 0) & (b.angles < 2 * np.pi))


def _region_bonds(problem):
    """Open bonds of the regions of the 7x7 scheme (shape bookkeeping)."""
    lat = problem.circuit.lattice
    cuts = set(problem.cut_edges)
    regions = {"A": lambda r, c: r < 3 and c < 3, "B": lambda r, c: r < 3 and c >= 3,
               "C": lambda r, c: r >= 3 and c < 3, "D": lambda r, c: r >= 3 and c >= 3}
    out = {}
    for name, f in regions.items():
        qs = {q for q, (r, c) in enumerate(lat.coords) if f(r, c)}
        out[name] = sum(1 for k, (a, b) in enumerate(lat.edges)
                        if ((a in qs) != (b in qs)) and k not in cuts)
    return out


def test_7x7_regions_have_six_open_bonds():
    """SI A: two cuts split 7x7x(1+40+1) into A, B, C, D of 2^(6x5) entries each
    and 2^(2x5) paths."""
    p = c2_problem(0, t=40)
    assert _region_bonds(p) == {"A": 6, "B": 6, "C": 6, "D": 6}
    K = cz_counts(p.circuit)
    assert all(K[e] == 5 for e in p.cut_edges)
    assert 2 ** int(sum(K[e] for e in p.cut_edges)) == 2 ** 10
