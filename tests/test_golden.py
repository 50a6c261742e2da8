"""Checks against values printed in the paper (tests/golden/paper_values.json)."""
import json
import os

import numpy as np

from oracle import permute as PM
from qflex_inputs import c2_problem, cz_counts

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_golden_permutation_moves():
    g = GOLD["permutation_example"]
    rng = np.random.default_rng(3)
    x = rng.normal(size=(3,) * 7)
    cur = list(g["source"])
    y = x
    for kind, gamma, new in g["moves"]:
        y = PM.apply_move(y, cur, list(new), kind, gamma)
        cur = list(new)
    assert "".join(cur) == g["target"]
    assert np.array_equal(y, PM.permute(x, [g["source"].index(c) for c in g["target"]]))


def test_golden_bris70_sizes():
    g = GOLD["bris70_sizes"]
    uncut = 2 ** (g["uncut_rank"] * g["K"]) * g["bytes_per_entry"]
    assert uncut / 1e12 > g["min_terabytes"]
    assert 2 ** (g["n_cuts"] * g["K"]) == 2 ** 16
    assert 2 ** (g["cut_rank"] * g["K"]) == 2 ** 28


def test_golden_7x7_sizes():
    g = GOLD["grid7x7_d40_sizes"]
    p = c2_problem(0, t=g["t"])
    K = cz_counts(p.circuit)
    assert int(np.prod([2 ** int(K[e]) for e in p.cut_edges])) == g["n_paths"]
    assert 2 ** (6 * int(K[0])) == g["region_entries"]


def test_golden_frugal_acceptance():
    g = GOLD["frugal_acceptance"]
    for nc, acc, batches in g["cases"]:
        p = 1 - (1 - 1 / g["M"]) ** nc
        assert abs(p - acc) < 5e-5
        assert abs(1e6 / p - batches) / batches < 1e-3


def test_golden_bris70_plan_sizes():
    """The planner, on the 70-qubit diamond with four cuts of the A-B bonds,
    reaches exactly the sizes the paper states: 2^(4x4) paths and a largest
    intermediate of 2^(7x4) entries (down from rank 11 without cuts)."""
    from paper_1811_09599_gb300.api import Plan
    from qflex_inputs import diamond_problem
    g = GOLD["bris70_sizes"]
    prob = diamond_problem(32, 0)
    assert prob.n == 70 and len(prob.cut_edges) == g["n_cuts"]
    info = Plan(prob, "bf16x3", device=-1).info()
    assert info["n_slices"] == 2 ** (g["n_cuts"] * g["K"])
    assert info["max_tensor_elems"] == 2 ** (g["cut_rank"] * g["K"])


def test_region_split_contraction_matches_oracle():
    """The golden writer of the 7x7 depth 1+40+1 paths (tests/golden/
    make_c4_golden.py) cuts two more bonds itself and sums over them where
    they close; on the same lattice and region cuts at depths 1+8+1 and
    1+16+1 its per-path amplitudes equal oracle.network.slice_amplitudes."""
    import importlib.util
    from oracle import network as NW
    from qflex_inputs import random_bitstrings
    spec = importlib.util.spec_from_file_location(
        "make_c4_golden", os.path.join(os.path.dirname(__file__), "golden", "make_c4_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    for t in (8, 16):
        prob = c2_problem(3, t=t)
        bits = random_bitstrings(prob.n, 1, 17)[0]
        P = NW.n_slices(prob.circuit, prob.cut_edges)
        for s in (0, 1, P - 1):
            got = mod.region_split_amplitudes(prob, bits, s, log=None)
            ref = NW.slice_amplitudes(prob, bits, s)
            assert np.allclose(got, ref, rtol=1e-10, atol=1e-13 * np.max(np.abs(ref))), (t, s)
