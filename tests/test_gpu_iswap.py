"""GPU parity of iSWAP circuits (Methods, "Revised set of RQCs": CZ replaced by
iSWAP; Schmidt rank 4, so each iSWAP adds two bond bits).

Amplitudes against the oracle's state vector and contraction, per-slice
values against the oracle's slice contraction, angle gradients of rotation
+ iSWAP circuits against the oracle's state-vector adjoint, and one slice of
the full-size 7x7 depth 1+16+1 iSWAP network (bond dimension 16, the shapes
of the 1+32+1 CZ workload).
"""
import numpy as np
import pytest

from oracle import gradients as GR
from oracle import network as NW
from oracle import statevector as SV
from qflex_inputs import c2_problem, grid_problem, random_bitstrings
from tests.gpu_util import TOL, amp_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = ["fp32", "tf32x3", "bf16x3", "fp16x3"]
GTOL = {"fp32": 2e-5, "tf32x3": 2e-4, "bf16x3": 2e-4, "fp16x3": 2e-4}


@pytest.fixture(scope="module")
def api():
    from paper_1811_09599_gb300 import api
    api._lib.load(build_if_missing=True)
    return api


def _amps(api, prob, prec, bs, slices=None):
    plan = api.Plan(prob, prec, device=0)
    out = plan.amplitudes(torch.from_numpy(np.ascontiguousarray(bs)).cuda(), None, slices).cpu().numpy()
    plan.sync()
    return out


@pytest.mark.parametrize("prec", PRECS)
def test_iswap_4x4_full_tile_vs_statevector(api, prec):
    """4x4, 1+8+1 iSWAP (bond dimension 4), tile = all 16 qubits."""
    prob = grid_problem(4, 4, 8, 5, r0=2, c0=2, cuts=False, tile_rows=4, tile_cols=4,
                        two_qubit="ISWAP")
    bs = random_bitstrings(16, 1, 0)
    got = _amps(api, prob, prec, bs)
    ref = SV.amplitudes(prob.circuit, bs, prob.open_tile)
    assert amp_error(got, ref, 16) < TOL[prec]
    assert abs(np.sum(np.abs(got) ** 2) - 1.0) < 10 * TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_iswap_cut_grid_all_and_single_slices(api, prec):
    """4x5, 1+16+1 iSWAP (bond dimension 16), two cuts (256 slices), 4-qubit
    tile: the full sum against the state vector, single slices against the
    oracle's slice contraction (which pins the 2-bit bond order)."""
    prob = grid_problem(4, 5, 16, 2, r0=2, c0=2, cuts=True, tile_rows=2, tile_cols=2,
                        two_qubit="ISWAP")
    P = NW.n_slices(prob.circuit, prob.cut_edges)
    assert P == 256
    bs = random_bitstrings(prob.n, 2, 9)
    got = _amps(api, prob, prec, bs)
    ref = SV.amplitudes(prob.circuit, bs, prob.open_tile)
    assert amp_error(got, ref, prob.n) < TOL[prec]
    tensors = NW.all_grid_tensors(prob.circuit)
    for s in (1, 6, 201):
        g1 = _amps(api, prob, prec, bs[:1], [s])
        r1 = NW.slice_amplitudes(prob, bs[0], s, tensors=tensors)
        assert amp_error(g1, r1, prob.n, 1.0 / P) < TOL[prec], s


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_iswap_rotation_gradients_vs_adjoint(api, prec):
    """3x4, 1+16+1 rotations with iSWAPs (bond dimension 16), two cuts, 2-qubit
    tile: every angle's gradient against the state-vector adjoint (the
    reverse sweep applies the iSWAP halves as row vectors)."""
    prob = grid_problem(3, 4, 16, 4, r0=2, c0=2, cuts=True, tile_rows=1, tile_cols=2,
                        rotations=True, two_qubit="ISWAP")
    bs = random_bitstrings(prob.n, 2, 4)
    rng = np.random.default_rng(6)
    g = (rng.standard_normal((2, 4)) + 1j * rng.standard_normal((2, 4))).astype(np.complex128)
    plan = api.Plan(prob, prec, device=0)
    amps, grad = plan.amplitudes_grad(torch.from_numpy(bs).cuda(),
                                      torch.from_numpy(prob.circuit.angles).cuda(),
                                      torch.from_numpy(g).cuda(), None)
    plan.sync()
    ref_amps = SV.amplitudes(prob.circuit, bs, prob.open_tile)
    ref = GR.statevector_adjoint(prob.circuit, bs, prob.open_tile, g)
    assert amp_error(amps.cpu().numpy(), ref_amps, prob.n) < TOL[prec]
    scale = np.linalg.norm(g.reshape(-1)) * 0.5 * np.sqrt(2.0 ** -prob.n)
    assert np.max(np.abs(grad.cpu().numpy() - ref)) / scale < GTOL[prec]


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_iswap_7x7_full_size_sampled_slice(api, prec):
    """7x7, 1+16+1 iSWAP, two cuts (256 slices), 6-qubit tile: the launch
    shapes of the 1+32+1 CZ workload (2^12 x 2^12 x 2^12 GEMMs); one
    sampled slice of one bitstring against the oracle's slice contraction."""
    prob = c2_problem(0, t=16, two_qubit="ISWAP")
    bs = random_bitstrings(prob.n, 1, 77)
    got = _amps(api, prob, prec, bs, [37])
    ref = NW.slice_amplitudes(prob, bs[0], 37)
    assert amp_error(got, ref, prob.n, 1.0 / 256) < TOL[prec]
