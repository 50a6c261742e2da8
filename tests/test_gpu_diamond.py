"""Bristlecone-like diamond (Methods "Cutting indexes": four cuts of 2^4,
regions A and B per path, path-independent C holding the open tile).

Small diamonds: full sums against the state vector, every slice and a
fraction-f sum against the oracle.  The 70-qubit diamond at depth 1+32+1:
one path (2^28-entry intermediates, 256-amplitude tile) against the oracle's
contraction of the same path, and the FP64 GPU norm of the tile amplitudes.
"""
import numpy as np
import pytest

from oracle import network as NW
from oracle import selection as SEL
from oracle import statevector as SV
from qflex_inputs import diamond_problem, random_bitstrings
from tests.gpu_util import TOL, amp_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1811_09599_gb300 import api
    api._lib.load(build_if_missing=True)
    return api


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_small_diamond_vs_statevector(api, prec):
    prob = diamond_problem(16, 3, size=6, n_cuts=1)          # 16 qubits, 8-qubit tile
    bs = random_bitstrings(prob.n, 2, 3)
    plan = api.Plan(prob, prec, device=0)
    got = plan.amplitudes(torch.from_numpy(bs).cuda()).cpu().numpy()
    ref = SV.amplitudes(prob.circuit, bs, prob.open_tile)
    assert amp_error(got, ref, prob.n) < TOL[prec]
    P = plan.n_slices
    for s in range(P):
        g1 = plan.amplitudes(torch.from_numpy(bs[:1]).cuda(), None, [s]).cpu().numpy()
        assert amp_error(g1, NW.slice_amplitudes(prob, bs[0], s), prob.n, 1.0 / P) < TOL[prec]


def test_diamond30_fraction_vs_oracle(api):
    prob = diamond_problem(24, 5, size=8, n_cuts=2)          # 30 qubits, 64 paths
    bs = random_bitstrings(prob.n, 1, 5)
    plan = api.Plan(prob, "bf16x3", device=0)
    P = plan.n_slices
    sel = plan.select_slices(0.25, 9)
    assert list(sel) == SEL.select_slices(P, 0.25, 9)
    got = plan.amplitudes(torch.from_numpy(bs).cuda(), None, sel).cpu().numpy()
    ref = NW.amplitudes(prob, bs, sel)
    assert amp_error(got, ref, prob.n, len(sel) / P) < TOL["bf16x3"]


# The 70-qubit diamond's plan runs 44 tensor-core products (36 on the 7x7
# grid): bf16 hi + lo operands (16 significand bits) measured 1.3e-4 here,
# so a bf16x3 plan of this length stores its planes as scaled fp16 hi + lo
# (22 bits; plane_format 3), and every precision keeps its bound.
BRIS70_TOL = dict(TOL)


def test_bris70_full_size_path(api):
    prob = diamond_problem(32, 0)                           # 70 qubits, 4 cuts
    bs = random_bitstrings(prob.n, 1, 77)
    s = 12345
    ref = NW.slice_amplitudes(prob, bs[0], s)
    errs = {}
    for prec in ("bf16x3", "tf32x3", "fp32", "fp16x3"):
        plan = api.Plan(prob, prec, device=0)
        got = plan.amplitudes(torch.from_numpy(bs).cuda(), None, [s])
        errs[prec] = amp_error(got.cpu().numpy(), ref, prob.n, 1.0 / 65536)
        nrm = api.norm(got).item()
        assert abs(nrm - float(np.sum(np.abs(ref) ** 2))) < 1e-3 * nrm
        plan.sync()
        plan.close()
    for prec, e in errs.items():
        assert e < BRIS70_TOL[prec], (prec, errs)


def test_bris70_tied_cuts_path(api):
    """Four cuts of the 70-qubit diamond of which two, (56, 62) and
    (56, 57), have their CZ projector halves in one diagonal stretch of
    qubit 56 (their bits are tied: 4,096 of the 2^16 paths are nonzero),
    with the search's ordering for them (2^28-entry limit): one path that
    does not vanish identically against the oracle's contraction of the same
    path with the same cuts and ordering; a path that vanishes identically
    gives exact zeros."""
    from qflex_inputs.problems import Problem
    d = diamond_problem(32, 0)
    ei = d.circuit.lattice.edge_index
    assert ei[(56, 62)] == 101 and ei[(56, 57)] == 100
    r = api.search_ordering(Problem(d.circuit, [101, 100, 11, 22], d.open_tile, None), 1 << 28, 0, trials=8, seed=0)
    assert r["fits"] and r["n_slices"] == 65536 and r["n_nonzero_slices"] == 4096
    prob = Problem(d.circuit, r["cuts"], d.open_tile, r["ordering"])
    bs = random_bitstrings(prob.n, 1, 78)
    nz = NW.nonzero_slices(prob.circuit, prob.cut_edges)      # paths that do not vanish identically
    s = nz[int(np.random.default_rng(4321).integers(len(nz)))]
    ref = NW.slice_amplitudes(prob, bs[0], s)
    plan = api.Plan(prob, "bf16x3", device=0)
    assert plan.info()["plane_format"] == 3          # long chain: scaled fp16 planes
    got = plan.amplitudes(torch.from_numpy(bs).cuda(), None, [s])
    plan.sync()
    nrm = api.norm(got).item()
    assert abs(nrm - float(np.sum(np.abs(ref) ** 2))) < 1e-3 * nrm
    # a kept path carries 1/len(nz) of the norm (not 1/65536): that sets
    # the floor of the relative error
    assert amp_error(got.cpu().numpy(), ref, prob.n, 1.0 / len(nz)) < BRIS70_TOL["bf16x3"]
    assert list(plan.nonzero_slices()) == nz
    if len(nz) < 65536:
        z = min(set(range(65536)) - set(nz))
        assert NW.structurally_zero(prob.circuit, prob.cut_edges, z)
        assert torch.count_nonzero(plan.amplitudes(torch.from_numpy(bs).cuda(), None, [z])).item() == 0
    plan.close()
