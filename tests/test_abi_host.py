"""C-ABI checks that need no GPU: symbols, host-only plans, validation errors."""
import re
import os

import numpy as np
import pytest

from oracle import network as NW
from oracle import selection as SEL
from qflex_inputs import c2_problem, c4_problem, grid_problem, random_circuit, grid_lattice
from qflex_inputs.problems import Problem

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "qflex.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qflex_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "qflex_amplitudes" in names and "qflex_permute" in names
    for n in names:
        assert hasattr(lib, n), n
    from paper_1811_09599_gb300._lib import SIGNATURES
    assert sorted(s[0] for s in SIGNATURES) == names


def test_abi_version(lib):
    assert lib.qflex_abi_version() == 4


@pytest.fixture
def Plan():
    from paper_1811_09599_gb300.api import Plan
    return Plan


@pytest.fixture
def api_mod():
    from paper_1811_09599_gb300 import api
    return api


def test_host_plan_7x7_d40_sizes(Plan):
    """SI A: 7x7x(1+40+1) with two cuts has 2^(2x5) paths and regions of 2^(6x5)."""
    p = Plan(c4_problem(0), "bf16x3", device=-1)
    info = p.info()
    assert info["n_slices"] == 1024
    assert info["max_tensor_elems"] == 2 ** 30
    assert info["n_open"] == 6 and info["n_qubits"] == 49


def test_host_plan_reuse_counts(Plan):
    """A is built once per bitstring, B/pD/AB once per right-cut value, the
    rest per slice (SI A's reuse of path-independent tensors)."""
    prob = c2_problem(0)
    p = Plan(prob, "fp32", device=-1)
    c1 = p.cost(1)
    # once: A (8 steps), B's (0,6)+(1,6) and pD's (6,6)+(5,6)+(4,6) (they touch
    # no cut bond: the paper's partial tensors pB / ppD)
    once = 8 + 1 + 2
    per_right = 10 + 9 + 1       # rest of B, rest of pD, AB
    per_slice = 4 + 1 + 12       # D column, ABD, region C
    assert c1["steps_executed"] == once + 16 * per_right + 256 * per_slice
    assert p.cost(3)["steps_executed"] == 3 * c1["steps_executed"]
    # AB and ABD are 2^12 x 2^12 x 2^12 complex GEMMs at K_e = 4
    assert c1["largest_gemm_cmacs"] == 2.0 ** 36


def test_select_slices_matches_oracle(Plan):
    p = Plan(c2_problem(0), "fp32", device=-1)
    for f, seed in ((0.01, 1), (0.1, 42), (0.5, 7), (1.0, 3)):
        assert list(p.select_slices(f, seed)) == SEL.select_slices(256, f, seed)


def test_host_plan_refuses_compute(Plan):
    import torch
    from paper_1811_09599_gb300 import QFlexError
    p = Plan(c2_problem(0), "fp32", device=-1)
    from paper_1811_09599_gb300._lib import check
    with pytest.raises(QFlexError) as e:
        check(p.lib.qflex_amplitudes(p.handle, None, None, 0, None, 0, None, None))
    assert "UNSUPPORTED" in str(e.value)
    with pytest.raises(QFlexError) as e:
        p.profile_shapes()
    assert "UNSUPPORTED" in str(e.value)


def test_validation_errors(Plan):
    from paper_1811_09599_gb300 import QFlexError
    prob = grid_problem(3, 3, 8, 0, r0=1, c0=1, cuts=False, tile_rows=1, tile_cols=1)
    # CZ on a non-edge
    bad = grid_problem(3, 3, 8, 0, r0=1, c0=1, cuts=False, tile_rows=1, tile_cols=1)
    for g in bad.circuit.gates:
        if g.kind == "CZ":
            g.q0, g.q1 = 0, 8
            break
    with pytest.raises(QFlexError, match="CIRCUIT"):
        Plan(bad, "fp32", device=-1)
    # ordering that leaves two tensors
    short = Problem(prob.circuit, [], prob.open_tile, prob.ordering[:-1])
    with pytest.raises(QFlexError, match="PLAN"):
        Plan(short, "fp32", device=-1)
    # ordering naming an absorbed tensor
    dup = Problem(prob.circuit, [], prob.open_tile, prob.ordering + [prob.ordering[0]])
    with pytest.raises(QFlexError, match="PLAN"):
        Plan(dup, "fp32", device=-1)
    # workspace budget
    with pytest.raises(QFlexError, match="PLAN"):
        Plan(c2_problem(0), "fp32", device=-1, workspace_bytes_max=1 << 20)
    # slice id out of range
    p = Plan(c2_problem(0), "fp32", device=-1)
    with pytest.raises(QFlexError, match="ARG"):
        p.cost(1, [256])
    # repeated tile qubit
    rep = Problem(prob.circuit, [], [1, 1], prob.ordering)
    with pytest.raises(QFlexError, match="ARG"):
        Plan(rep, "fp32", device=-1)


def test_default_ordering_and_rotation_circuits(Plan):
    circ = random_circuit(grid_lattice(3, 3), 16, 2, rotations=True)
    p = Plan(Problem(circ, [], [0, 4], None), "tf32x3", device=-1)
    info = p.info()
    assert info["n_params"] == circ.n_params and info["n_steps"] == 8


def test_iswap_plan_costs_what_cz_at_twice_the_depth(Plan):
    """Methods, "Revised set of RQCs": an iSWAP circuit of depth 1+t/2+1 costs
    what a CZ circuit of depth 1+t+1 costs (each iSWAP adds 2 bond bits).  The
    planner's own accounting of the 7x7 two-cut workload agrees exactly."""
    cz = Plan(c2_problem(0, t=32), "bf16x3", device=-1)
    isw = Plan(c2_problem(0, t=16, two_qubit="ISWAP"), "bf16x3", device=-1)
    a, b = cz.info(), isw.info()
    for k in ("n_slices", "max_tensor_elems", "n_steps", "n_tc_steps"):
        assert a[k] == b[k], k
    # the workspace also holds the compiled gate lines (578 gates vs 1050)
    assert abs(a["workspace_bytes"] - b["workspace_bytes"]) < 64 << 10
    ca, cb = cz.cost(1), isw.cost(1)
    for k in ("steps_executed", "largest_gemm_cmacs", "cmacs", "tc_mma_flops", "permute_bytes", "launches"):
        assert ca[k] == cb[k], k


def test_iswap_validation(Plan):
    from paper_1811_09599_gb300 import QFlexError
    # an iSWAP on a pair that is not a lattice edge
    bad = grid_problem(3, 3, 8, 0, r0=1, c0=1, cuts=False, tile_rows=1, tile_cols=1, two_qubit="ISWAP")
    for g in bad.circuit.gates:
        if g.kind == "ISWAP":
            g.q0, g.q1 = 0, 8
            break
    with pytest.raises(QFlexError, match="CIRCUIT"):
        Plan(bad, "fp32", device=-1)
    # more than 20 bond bits on one edge: 11 iSWAPs (22 bits)
    deep = random_circuit(grid_lattice(2, 2), 88, 0, two_qubit="ISWAP")
    with pytest.raises(QFlexError, match="PLAN"):
        Plan(Problem(deep, [], [], None), "fp32", device=-1)


def test_fidelity_samples_argument_checks():
    """qflex_fidelity_samples validates on the host before any device work."""
    import ctypes as C
    from paper_1811_09599_gb300 import _lib
    lib = _lib.load()
    n_exact = C.c_int64(-1)
    tile = (C.c_int32 * 2)(3, 3)
    # repeated tile qubit, fidelity outside [0, 1], too many tile qubits
    assert lib.qflex_fidelity_samples(None, None, 0, tile, 2, 8, 0.5, 1, 4, None, None,
                                      C.byref(n_exact), None) == 1
    tile = (C.c_int32 * 2)(3, 4)
    assert lib.qflex_fidelity_samples(None, None, 0, tile, 2, 8, 1.5, 1, 4, None, None,
                                      C.byref(n_exact), None) == 1
    assert lib.qflex_fidelity_samples(None, None, 0, tile, 31, 40, 0.5, 1, 4, None, None,
                                      C.byref(n_exact), None) == 1
    # no draws: nothing to do
    assert lib.qflex_fidelity_samples(None, None, 0, tile, 2, 8, 0.5, 1, 0, None, None,
                                      C.byref(n_exact), None) == 0 and n_exact.value == 0


def test_plan_steps_agree_with_cost(Plan):
    """qflex_plan_steps: per-step shapes and executions add up to the
    host cost replay, and the execution counts follow SI A's reuse (the
    4096^3 ABD product once per slice, AB once per right-cut value)."""
    p = Plan(c2_problem(0), "bf16x3", device=-1)
    for n_bs, ids in ((1, None), (3, [5, 6, 200])):
        steps = p.steps(n_bs, ids)
        c = p.cost(n_bs, ids)
        assert len(steps) == p.info()["n_steps"]
        assert sum(s["runs"] for s in steps) == c["steps_executed"]
        assert sum(s["M"] * s["N"] * s["K"] * s["runs"] for s in steps) == c["cmacs"]
        assert sum(s["M"] * s["N"] * s["K"] * s["runs"] for s in steps
                   if s["kernel"] == "tensor_cores") == c["tc_cmacs"]
        assert sum(16 * (s["a_builds"] * s["M"] + s["b_builds"] * s["N"]) * s["K"]
                   for s in steps) == c["permute_bytes"]
    big = [s for s in p.steps(1) if (s["M"], s["N"], s["K"]) == (4096, 4096, 4096)]
    assert sorted(s["runs"] for s in big) == [16, 256]
    assert all(s["kernel"] == "tensor_cores" for s in big)
    # both ABD operands are written by their producers' epilogues (fusion)
    abd = [s for s in big if s["runs"] == 256][0]
    assert abd["a_fused"] and abd["b_fused"] and abd["a_builds"] == 0 and abd["b_builds"] == 0
    # without fusion (plain FP32 plan): AB's output order is already ABD's
    # operand layout (legs the consumer contracts go last), so it is read in
    # place; pD (changes once per right-cut value) keeps its permuted operand
    # for the first D-column absorb: built 16 times, not 256
    f = Plan(c2_problem(0), "fp32", device=-1)
    st32 = f.steps(1)
    abd32 = [s for s in st32 if (s["M"], s["N"], s["K"], s["runs"]) == (4096, 4096, 4096, 256)][0]
    assert abd32["a_direct"] and abd32["b_builds"] == 256
    d0 = [s for s in st32 if (s["M"], s["N"], s["K"]) == (1 << 20, 16, 16)][0]
    assert d0["a_cached"] and d0["a_builds"] == 16 and d0["runs"] == 256
    assert all(s["kernel"] != "tensor_cores" for s in Plan(c2_problem(0), "fp32", device=-1).steps(1))


def _constrained_problems():
    """Problems whose cuts leave paths that vanish identically (projector
    halves in one diagonal stretch), and one where none do."""
    from qflex_inputs import diamond_problem
    rot = grid_problem(4, 5, 24, 3, r0=2, c0=2, cuts=True, tile_rows=2, tile_cols=2, rotations=True)
    circ = random_circuit(grid_lattice(3, 3), 16, 0)
    ei = circ.lattice.edge_index
    corr = Problem(circ, [ei[(4, 5)], ei[(4, 7)], ei[(1, 2)]], [8], None)
    d = diamond_problem(32, 0)
    bris = Problem(d.circuit, [101, 100, 11, 22], d.open_tile, None)   # two bonds of qubit 56
    isw = grid_problem(4, 5, 16, 8, r0=2, c0=2, cuts=True, tile_rows=2, tile_cols=2, two_qubit="ISWAP")
    return [rot, corr, bris, c2_problem(0), isw]


def test_nonzero_slices_match_oracle(Plan):
    """qflex_nonzero_slices / qflex_select_nonzero_slices against the
    oracle's projector rule, and the plan info count."""
    from paper_1811_09599_gb300 import QFlexError
    for prob in _constrained_problems():
        p = Plan(prob, "bf16x3", device=-1)
        ref = NW.nonzero_slices(prob.circuit, prob.cut_edges)
        assert list(p.nonzero_slices()) == ref
        assert p.info()["n_nonzero_slices"] == len(ref)
        for f, seed in ((0.01, 2026), (0.3, 5), (1.0, 1)):
            want = sorted(ref[i] for i in SEL.select_slices(len(ref), f, seed))
            assert list(p.select_slices(f, seed, nonzero=True)) == want
    import ctypes as C
    p = Plan(_constrained_problems()[1], "fp32", device=-1)
    n = C.c_int64()
    assert p.lib.qflex_nonzero_slices(p.handle, 0, None, 0, C.byref(n)) != 0   # capacity too small
    assert n.value == p.info()["n_nonzero_slices"] < p.n_slices
    with pytest.raises(QFlexError, match="ARG"):
        from paper_1811_09599_gb300._lib import check
        check(p.lib.qflex_nonzero_slices(p.handle, 0, None, 0, None))


def test_vanishing_paths_are_skipped_in_the_schedule(Plan):
    """The cost replay (the executor's schedule) runs nothing for a path that
    vanishes identically: all paths cost what the nonzero ones cost, and a
    list of vanishing paths only builds the grid tensors."""
    prob = _constrained_problems()[0]
    p = Plan(prob, "bf16x3", device=-1)
    nz = list(p.nonzero_slices())
    zero = sorted(set(range(p.n_slices)) - set(nz))
    assert len(zero) > 0
    assert p.cost(2) == p.cost(2, nz)
    c0 = p.cost(1, zero[:5])
    assert c0["cmacs"] == 0 and c0["steps_executed"] == 0
    assert p.cost(1, sorted(nz[:3] + zero[:3])) == p.cost(1, nz[:3])


def test_selftest_timeout_argument_checks(lib):
    """qflex_device_selftest_timeout rejects a bad device or limit before
    touching a GPU."""
    import ctypes as C
    v = C.c_int32()
    assert lib.qflex_device_selftest_timeout(-1, C.c_uint64(10_000_000), C.byref(v)) == 1
    assert lib.qflex_device_selftest_timeout(0, C.c_uint64(10), C.byref(v)) == 1
    assert lib.qflex_device_selftest_timeout(0, C.c_uint64(10 ** 10), C.byref(v)) == 1
    assert lib.qflex_device_selftest_timeout(0, C.c_uint64(10_000_000), None) == 1


def _plain_work(prob):
    """Complex MACs of one bitstring, counted from the definition: each
    ordering step multiplies 2^(a + b - s) (a, b: index bits of the two
    groups' tensors, s: bits they share) and runs once per change of the
    values of the cuts touching its group along the ascending list of
    paths that do not vanish identically (the oracle's list)."""
    circ = prob.circuit
    K = NW.bond_exponents(circ)
    cut = list(prob.cut_edges)
    nz = NW.nonzero_slices(circ, cut)
    vals = [NW.slice_values(circ, cut, s) for s in nz]

    def bits_of(group):
        legs = {}
        for e, (a, b) in enumerate(circ.edges):
            if K[e] and e not in cut and ((a in group) != (b in group)):
                legs[("e", e)] = int(K[e])
        for q in group:
            if q in prob.open_tile:
                legs[("o", q)] = 1
        return legs

    def runs(group):
        dep = [e for e in cut if circ.edges[e][0] in group or circ.edges[e][1] in group]
        count, prev = 0, None
        for v in vals:
            key = tuple(v[e] for e in dep)
            if key != prev:
                count += 1
            prev = key
        return count

    groups = {q: {q} for q in range(circ.n)}
    total = 0
    for dst, src in prob.ordering:
        la, lb = bits_of(groups[dst]), bits_of(groups[src])
        s = sum(v for k, v in la.items() if k in lb)
        merged = groups[dst] | groups.pop(src)
        total += runs(merged) * 2 ** (sum(la.values()) + sum(lb.values()) - s)
        groups[dst] = merged
    return total


def test_cost_replay_matches_the_plain_count(Plan, api_mod):
    """qflex_plan_cost's complex MACs (bench.py's TFLOP/s numerator) equal
    the count from the definition, with reuse across paths and vanishing
    paths skipped: the 7x7 region plan, a rotation circuit whose cuts leave
    vanishing paths, and a searched plan with tied cut pairs."""
    rot = grid_problem(4, 5, 24, 3, r0=2, c0=2, cuts=True, tile_rows=2, tile_cols=2, rotations=True)
    small = grid_problem(4, 5, 24, 7, r0=2, c0=2, cuts=False, tile_rows=2, tile_cols=2)
    r = api_mod.search_ordering(Problem(small.circuit, [], small.open_tile, None), 1 << 12, 4, trials=16)
    searched = Problem(small.circuit, r["cuts"], small.open_tile, r["ordering"])
    for prob in (c2_problem(0), rot, searched):
        p = Plan(prob, "bf16x3", device=-1)
        assert p.cost(1)["cmacs"] == _plain_work(prob)


def test_multi_problem_plan_matches_single_plans(Plan):
    """qflex_plan_create over several problems (uneven rotation circuits,
    two grids with cuts and tiles): each problem's info, cost and schedule
    equal those of a plan of that problem alone; the flat-array layout of a
    call follows the problems' sizes; a bad problem index is an argument
    error and a bad problem is reported by its index."""
    from paper_1811_09599_gb300._lib import QFlexError
    from qflex_inputs import grid_problem, rotation_batch
    probs = rotation_batch(6, 3) + [grid_problem(4, 5, 32, 5, r0=2, c0=2, cuts=True, tile_rows=2, tile_cols=2),
                                   c2_problem(0)]
    multi = Plan(probs, "bf16x3", device=-1)
    assert multi.n_problems == len(probs)
    tot = 0
    for k, pr in enumerate(probs):
        one = Plan(pr, "bf16x3", device=-1)
        a, b = multi.info(k), one.info()
        assert a["n_problems"] == len(probs) and b["n_problems"] == 1
        for key in ("n_slices", "n_qubits", "n_params", "n_open", "n_steps", "max_tensor_elems", "n_tc_steps",
                    "n_nonzero_slices", "plane_format"):
            assert a[key] == b[key], (k, key)
        assert a["problem_workspace_bytes"] == b["workspace_bytes"]
        tot += b["workspace_bytes"]
        assert multi.cost(2, None, k) == one.cost(2)
        assert multi.steps(2, None, k) == one.steps(2)
    assert multi.info(0)["workspace_bytes"] >= tot
    lay = multi.layout(3)
    assert lay["bits"][-1] == 3 * sum(p.n for p in probs)
    assert lay["params"][-1] == sum(p.circuit.n_params for p in probs)
    assert lay["amps"][-1] == 3 * sum(1 << len(p.open_tile) for p in probs)
    with pytest.raises(QFlexError, match="ARG"):
        multi.info(len(probs))
    bad = grid_problem(3, 3, 8, 1, cuts=False, tile_rows=0)
    bad.ordering = bad.ordering[:-1]                       # does not contract to one tensor
    with pytest.raises(QFlexError, match="problem 2"):
        Plan(probs[:2] + [bad], "fp32", device=-1)


def test_bf16x3_plane_format_by_chain_length(Plan):
    """QFLEX_BF16X3 keeps bf16 planes up to 36 tensor-core steps (the 7x7
    depth-32 region plan) and stores longer chains (7x7 depth 40, the
    70-qubit diamond) as scaled fp16 planes; the other precisions keep theirs."""
    from qflex_inputs import c4_problem, diamond_problem
    fmt = lambda pr, prec: Plan(pr, prec, device=-1).info()
    c2, c4, d = fmt(c2_problem(0), "bf16x3"), fmt(c4_problem(0), "bf16x3"), fmt(diamond_problem(32, 0), "bf16x3")
    assert (c2["n_tc_steps"], c2["plane_format"]) == (36, 2)
    assert c4["n_tc_steps"] > 36 and c4["plane_format"] == 3
    assert d["n_tc_steps"] > 36 and d["plane_format"] == 3
    assert fmt(diamond_problem(32, 0), "tf32x3")["plane_format"] == 1
    assert fmt(diamond_problem(32, 0), "fp16x3")["plane_format"] == 3
    assert fmt(c2_problem(0), "fp32")["plane_format"] == 0


def test_wide_mma_choice(Plan):
    """Split tensor-core products take one MMA of width 2 bn ([hi.hi | hi.lo])
    plus one of width bn per k-step for 64-wide tiles and, with 128-wide
    tiles, for K >= 256; otherwise three of width bn.  In the 7x7 1+32+1
    plan that puts the 4096^3 products and the K = 256 region absorbs on the
    wide form and the K = 16 products on the three-MMA form; unsplit
    precisions never use it."""
    for prec in ("bf16x3", "fp16x3", "tf32x3", "bf16", "fp32"):
        steps = Plan(c2_problem(0), prec, device=-1).steps(1)
        for s in steps:
            split = prec in ("bf16x3", "fp16x3", "tf32x3")
            want = s["kernel"] == "tensor_cores" and split and (s["bn"] == 64 or s["K"] >= 256)
            assert s["tc_wide"] == int(want), (prec, s["M"], s["N"], s["K"], s["bn"])
        if prec == "bf16x3":
            big = [s for s in steps if (s["M"], s["N"], s["K"]) == (4096, 4096, 4096)]
            absorb = [s for s in steps if (s["M"], s["N"], s["K"]) == (65536, 256, 256)]
            assert big and absorb
            k16 = [s for s in steps if s["kernel"] == "tensor_cores" and s["K"] == 16 and s["bn"] == 128]
            assert k16 and all(s["tc_wide"] for s in big + absorb) and not any(s["tc_wide"] for s in k16)
