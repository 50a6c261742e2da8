"""Automated cut and ordering search (qflex_search_ordering), on the host.

The paper picks cuts and contraction orders by hand (Methods, "Cutting
indexes"; SI A).  The search must (a) return valid orderings that the
planner accepts, (b) estimate the work exactly as the executor counts it
(steps rerun only when a cut they depend on changes), (c) reach the exact
optimum of its move set on networks small enough for brute force, and
(d) find, for the 7x7 depth 1+32+1 grid and the 70-qubit diamond,
configurations of the paper's size class (256 and at most 2^16 nonzero
paths; tensors of at most 2^24 and 2^28 entries) with less work than the
region plans.
"""
import functools
import math

import pytest

from oracle import network as NW
from qflex_inputs import c2_problem, diamond_problem, grid_lattice, grid_problem, random_circuit
from qflex_inputs.circuits import two_qubit_counts
from qflex_inputs.problems import Problem


@pytest.fixture(scope="module")
def api():
    from paper_1811_09599_gb300 import api
    return api


def _bits(circ):
    """Bond bits per edge: 1 per CZ, 2 per iSWAP."""
    bits = [0] * len(circ.edges)
    idx = circ.lattice.edge_index
    for g in circ.gates:
        if g.kind in ("CZ", "ISWAP"):
            bits[idx[(min(g.q0, g.q1), max(g.q0, g.q1))]] += 1 if g.kind == "CZ" else 2
    return bits


def brute_force_min_work(circ, tile, cuts):
    """Least work over every sequence of contractions of tensors sharing a
    bond, with each step weighted by how often the executor runs it (once per
    change of the cuts it depends on, first cut most significant)."""
    bits = _bits(circ)
    n, E = circ.n, len(circ.edges)
    radix = [2 ** bits[e] for e in cuts]

    def legs_of(group):
        legs = {}
        for e, (a, b) in enumerate(circ.edges):
            if bits[e] == 0 or e in cuts:
                continue
            ina, inb = a in group, b in group
            if ina != inb:
                legs[e] = bits[e]
        for q in group:
            if q in tile:
                legs[E + q] = 1
        return legs

    def runs(group):
        dep = [i for i, e in enumerate(cuts) if circ.edges[e][0] in group or circ.edges[e][1] in group]
        return math.prod(radix[: max(dep) + 1]) if dep else 1

    @functools.lru_cache(maxsize=None)
    def best(state):
        groups = list(state)
        if len(groups) == 1:
            return 0.0
        out = math.inf
        for i in range(len(groups)):
            for j in range(i + 1, len(groups)):
                la, lb = legs_of(groups[i]), legs_of(groups[j])
                s = sum(v for k, v in la.items() if k in lb)
                if s == 0:
                    continue
                merged = groups[i] | groups[j]
                work = runs(merged) * 2.0 ** (sum(la.values()) + sum(lb.values()) - s)
                rest = frozenset(g for k, g in enumerate(groups) if k not in (i, j)) | {merged}
                out = min(out, work + best(rest))
        return out

    return best(frozenset(frozenset([q]) for q in range(n)))


@pytest.mark.parametrize("rows,cols,t,tile,ncut", [(2, 3, 16, [5], 0), (3, 3, 16, [8], 1), (2, 4, 24, [6, 7], 1)])
def test_search_reaches_brute_force_optimum(api, rows, cols, t, tile, ncut):
    circ = random_circuit(grid_lattice(rows, cols), t, 3)
    cuts = [len(circ.edges) // 2] if ncut else []
    opt = brute_force_min_work(circ, tile, cuts)
    r = api.search_ordering(Problem(circ, cuts, tile, None), 1 << 40, 0, trials=256, seed=1)
    assert r["fits"]
    assert r["cmacs_per_bitstring"] == pytest.approx(opt, rel=1e-12)


@pytest.mark.parametrize("rotations", [False, True])
def test_search_work_model_matches_planner(api, rotations):
    """The search's work per bitstring equals the planner's cost replay of
    the same cuts and ordering (same reuse rule); with rotation gates the
    cuts leave paths that vanish identically (R_Z is diagonal), which both
    skip."""
    from paper_1811_09599_gb300.api import Plan
    p = grid_problem(4, 5, 24, 3, r0=2, c0=2, cuts=True, tile_rows=2, tile_cols=2, rotations=rotations)
    r = api.search_ordering(Problem(p.circuit, p.cut_edges, p.open_tile, None), 1 << 20, 0, trials=16)
    plan = Plan(Problem(p.circuit, r["cuts"], p.open_tile, r["ordering"]), "bf16x3", device=-1)
    assert plan.cost(1)["cmacs"] == pytest.approx(r["cmacs_per_bitstring"], rel=1e-12)
    assert math.log2(plan.info()["max_tensor_elems"]) <= r["log2_max_tensor"]
    assert r["n_nonzero_slices"] == plan.info()["n_nonzero_slices"]
    assert (r["n_nonzero_slices"] < r["n_slices"]) == rotations


def test_search_7x7_finds_tied_cut_plan(api):
    """7x7, 1+32+1, no cuts given, limit 2^24 entries, up to four new cuts:
    the search keeps the paper's 256 paths and tensor limit but reaches them
    with three cuts, two of whose bonds share a diagonal stretch of one
    qubit's projector halves (their bits are tied, so 256 of the 4,096 paths
    are nonzero), at under 0.3x the hand plan's work (both counted by the
    planner's cost replay).  The region ordering with the paper's two cuts
    is what the search finds when no new cut is allowed, within 1.15x."""
    from paper_1811_09599_gb300.api import Plan
    p = c2_problem(0)
    r = api.search_ordering(Problem(p.circuit, [], p.open_tile, None), 1 << 24, 4, trials=32, seed=0)
    assert r["fits"] and r["n_nonzero_slices"] == 256 and r["log2_max_tensor"] <= 24
    assert r["cuts"] == [32, 33, 80] and r["n_slices"] == 4096   # also pinned in the GPU test
    hand = Plan(p, "bf16x3", device=-1).cost(1)["cmacs"]
    found = Plan(Problem(p.circuit, r["cuts"], p.open_tile, r["ordering"]), "bf16x3", device=-1)
    assert found.info()["max_tensor_elems"] <= 1 << 24
    assert found.cost(1)["cmacs"] == pytest.approx(r["cmacs_per_bitstring"], rel=1e-12)
    assert found.cost(1)["cmacs"] <= 0.3 * hand
    # the two tied bonds: projector halves of one qubit with no non-diagonal gate between
    runs, _ = NW.projector_runs(p.circuit, r["cuts"])
    assert any(len({e for e, _ in m}) == 2 for m in runs)
    # the paper's cuts, ordering searched
    q = api.search_ordering(Problem(p.circuit, p.cut_edges, p.open_tile, None), 1 << 24, 0, trials=32, seed=0)
    assert q["fits"] and q["n_slices"] == 256 and q["cmacs_per_bitstring"] <= 1.15 * hand
    # deterministic for a given seed
    again = api.search_ordering(Problem(p.circuit, [], p.open_tile, None), 1 << 24, 4, trials=32, seed=0)
    assert again["cuts"] == r["cuts"] and again["ordering"] == r["ordering"]


def test_search_bristlecone_70(api):
    """Bris-70, 1+32+1, limit 2^28 entries: four cuts (2^16 paths), the
    configuration the paper states for this lattice; the search picks two
    pairs of bonds with tied projector bits (256 nonzero paths) and needs
    under 1% of the region plan's work for all paths."""
    from paper_1811_09599_gb300.api import Plan
    d = diamond_problem(32, 0)
    r = api.search_ordering(Problem(d.circuit, [], d.open_tile, None), 1 << 28, 4, trials=8, seed=0)
    assert r["fits"] and r["cuts"] == [100, 101, 72, 73] and r["n_slices"] == 65536
    assert r["n_nonzero_slices"] == 256            # two pairs of tied bonds
    hand = Plan(d, "bf16x3", device=-1).cost(1)["cmacs"]
    found = Plan(Problem(d.circuit, r["cuts"], d.open_tile, r["ordering"]), "bf16x3", device=-1)
    assert found.info()["max_tensor_elems"] <= 1 << 28
    assert found.cost(1)["cmacs"] <= 0.01 * hand


def test_searched_tied_cuts_sum_to_the_state_vector(api):
    """4x5, 1+24+1, limit 2^12: the search cuts tied pairs of bonds, most
    paths vanish identically, and the oracle's sum over the others, with
    the searched cuts and ordering, is the state-vector amplitude."""
    from oracle import statevector as SV
    from qflex_inputs import random_bitstrings
    p = grid_problem(4, 5, 24, 7, r0=2, c0=2, cuts=False, tile_rows=2, tile_cols=2)
    r = api.search_ordering(Problem(p.circuit, [], p.open_tile, None), 1 << 12, 4, trials=16)
    assert r["fits"] and r["n_nonzero_slices"] < r["n_slices"]
    prob = Problem(p.circuit, r["cuts"], p.open_tile, r["ordering"])
    nz = NW.nonzero_slices(prob.circuit, prob.cut_edges)
    assert len(nz) == r["n_nonzero_slices"]
    bs = random_bitstrings(p.n, 1, 5)
    got = NW.amplitudes(prob, bs, nz)
    assert abs(got - SV.amplitudes(p.circuit, bs, p.open_tile)).max() < 1e-14


def test_search_8x9_three_cuts(api):
    """8x9 grid (72 qubits), 1+32+1, limit 2^28 entries: three cuts suffice
    (the paper's comparison with Bris-70, which needs four: Methods,
    "Simulation of Bristlecone compared to rectangular grids")."""
    circ = random_circuit(grid_lattice(8, 9), 32, 0)
    r = api.search_ordering(Problem(circ, [], [71], None), 1 << 28, 3, trials=4, seed=0)
    assert r["fits"] and len(r["cuts"]) <= 3 and r["log2_max_tensor"] <= 28


def test_search_limits_and_defaults(api):
    from paper_1811_09599_gb300 import QFlexError
    from paper_1811_09599_gb300.api import Plan
    p = grid_problem(4, 4, 16, 1, r0=2, c0=2, cuts=False, tile_rows=1, tile_cols=2)
    # an unreachable limit without new cuts: best effort returned, fits False
    r = api.search_ordering(Problem(p.circuit, [], p.open_tile, None), 1 << 4, 0)
    assert not r["fits"] and len(r["ordering"]) == p.n - 1
    # the planner's default (ordering = None) is a valid greedy ordering
    plan = Plan(Problem(p.circuit, [], p.open_tile, None), "fp32", device=-1)
    assert plan.info()["n_steps"] == p.n - 1
    with pytest.raises(QFlexError, match="ARG"):
        api.search_ordering(Problem(p.circuit, [3, 3], p.open_tile, None), 1 << 20, 0)
    assert sum(two_qubit_counts(p.circuit)) > 0
