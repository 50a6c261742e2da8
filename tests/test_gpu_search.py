"""GPU parity of plans whose cuts and ordering come from the automated search
(qflex_search_ordering) or the planner's default ordering, against the
oracle's state vector: the amplitude does not depend on how the network is
cut or ordered (Methods, "Cutting indexes")."""
import numpy as np
import pytest

from oracle import statevector as SV
from qflex_inputs import grid_problem, random_bitstrings
from qflex_inputs.problems import Problem
from tests.gpu_util import TOL, amp_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1811_09599_gb300 import api
    api._lib.load(build_if_missing=True)
    return api


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_searched_cuts_and_ordering_vs_statevector(api, prec):
    """4x5, 1+24+1 (bond dimension 8), 4-qubit tile; the search adds cuts
    until every tensor has at most 2^12 entries."""
    p = grid_problem(4, 5, 24, 7, r0=2, c0=2, cuts=False, tile_rows=2, tile_cols=2)
    r = api.search_ordering(Problem(p.circuit, [], p.open_tile, None), 1 << 12, 4, trials=16)
    assert r["fits"] and len(r["cuts"]) >= 1
    prob = Problem(p.circuit, r["cuts"], p.open_tile, r["ordering"])
    bs = random_bitstrings(p.n, 2, 3)
    plan = api.Plan(prob, prec, device=0)
    got = plan.amplitudes(torch.from_numpy(bs).cuda()).cpu().numpy()
    plan.sync()
    ref = SV.amplitudes(p.circuit, bs, p.open_tile)
    assert amp_error(got, ref, p.n) < TOL[prec]


def test_default_ordering_vs_statevector(api):
    """The planner's default ordering (ordering = None) with the region cuts."""
    p = grid_problem(4, 5, 16, 8, r0=2, c0=2, cuts=True, tile_rows=2, tile_cols=2, two_qubit="ISWAP")
    prob = Problem(p.circuit, p.cut_edges, p.open_tile, None)
    bs = random_bitstrings(p.n, 2, 4)
    plan = api.Plan(prob, "bf16x3", device=0)
    got = plan.amplitudes(torch.from_numpy(bs).cuda()).cpu().numpy()
    plan.sync()
    ref = SV.amplitudes(p.circuit, bs, p.open_tile)
    assert amp_error(got, ref, p.n) < TOL["bf16x3"]
