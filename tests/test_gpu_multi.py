"""One plan and one call over many independent problems (qflex_plan_create
with n_problems > 1).  The paper runs independent instances, paths and
batches as separate jobs of one cluster run (Methods, "Simulation of RQCs on
NASA HPC clusters"); here they are the problems of one plan, whose call
spreads them over the plan's streams (captured into one CUDA graph with
qflex_plan_use_graphs).  Each problem's result must be the one a plan of
that problem alone gives, and the oracle's."""
import numpy as np
import pytest

from oracle import gradients as GR
from oracle import statevector as SV
from qflex_inputs import c1_problem, grid_problem, random_bitstrings, rotation_batch
from tests.gpu_util import TOL, amp_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1811_09599_gb300 import api
    api._lib.load(build_if_missing=True)
    return api


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_rotation_batch_one_call_equals_separate_plans(api, prec):
    """24 uneven rotation circuits (4x4..6x6, depth 1+16..32+1), one
    amplitude and every angle gradient each, in one qflex_amplitudes_grad
    call (direct, captured, replayed): amplitudes bit for bit those of one
    plan per circuit, gradients equal up to the order of their FP64 atomic
    sums, the first two circuits of at most 20 qubits against the
    state-vector adjoint."""
    probs = rotation_batch(24, 0)
    bits = [random_bitstrings(p.n, 1, 5000 + i) for i, p in enumerate(probs)]
    flat_bits = torch.from_numpy(np.concatenate([b.reshape(-1) for b in bits])).cuda()
    flat_th = torch.from_numpy(np.concatenate([p.circuit.angles for p in probs])).cuda()
    multi = api.Plan(probs, prec, device=0)
    multi.use_graphs(True)
    n_par = sum(p.circuit.n_params for p in probs)
    g = torch.zeros((1, len(probs), 2), dtype=torch.float64, device="cuda")
    g[..., 0] = 1.0
    out = torch.empty((1, len(probs), 2), dtype=torch.float64, device="cuda")
    gout = torch.empty(n_par, dtype=torch.float64, device="cuda")
    for _ in range(3):
        amps, grad = multi.amplitudes_grad(flat_bits, flat_th, g, out=out, grad_out=gout)
    multi.sync()
    amps, grad = amps.cpu().numpy(), grad.cpu().numpy()
    lay = multi.layout(1)
    small = [k for k, p in enumerate(probs) if p.n <= 20][:2]   # state vectors of at most 2^20 entries
    assert len(small) == 2
    for k, p in enumerate(probs):
        one = api.Plan(p, prec, device=0)
        a1, g1 = one.amplitudes_grad(torch.from_numpy(bits[k]).cuda(), torch.from_numpy(p.circuit.angles).cuda(),
                                     torch.ones((1, 1), dtype=torch.complex128, device="cuda"))
        one.sync()
        a1, g1 = a1.cpu().numpy().reshape(-1), g1.cpu().numpy()
        assert np.array_equal(amps[lay["amps"][k]:lay["amps"][k + 1]], a1), k
        gk = grad[lay["params"][k]:lay["params"][k + 1]]
        assert np.max(np.abs(gk - g1)) <= 1e-12 * np.max(np.abs(g1)), k
        if k in small:
            ref = SV.amplitudes(p.circuit, bits[k], [])
            assert amp_error(a1, ref, p.n) < TOL[prec]
            gref = GR.statevector_adjoint(p.circuit, bits[k], [], np.ones((1, 1), dtype=np.complex128))
            tol = 2e-5 if prec == "fp32" else 2e-4
            assert np.max(np.abs(gk - gref)) / (0.5 * np.sqrt(2.0 ** -p.n)) < tol, k


def test_mixed_problems_one_call_vs_statevector(api):
    """A 4x4 circuit with its full 16-qubit tile, a 4x5 grid with two cuts
    and a 4-qubit tile, and a 4x4 circuit of single amplitudes, 2
    bitstrings each, in one qflex_amplitudes call (graph replay on the
    third call): every problem's amplitudes against the state vector."""
    probs = [c1_problem(0, full_tile=True),
             grid_problem(4, 5, 32, 5, r0=2, c0=2, cuts=True, tile_rows=2, tile_cols=2),
             c1_problem(3, full_tile=False)]
    n_bs = 2
    bits = [random_bitstrings(p.n, n_bs, 40 + i) for i, p in enumerate(probs)]
    flat = torch.from_numpy(np.concatenate([b.reshape(-1) for b in bits])).cuda()
    plan = api.Plan(probs, "bf16x3", device=0)
    plan.use_graphs(True)
    T = sum(1 << len(p.open_tile) for p in probs)
    out = torch.empty((n_bs, T, 2), dtype=torch.float64, device="cuda")
    for _ in range(3):
        amps = plan.amplitudes(flat, None, None, out=out)
    plan.sync()
    amps = amps.cpu().numpy()
    lay = plan.layout(n_bs)
    for k, p in enumerate(probs):
        got = amps[lay["amps"][k]:lay["amps"][k + 1]].reshape(n_bs, -1)
        ref = SV.amplitudes(p.circuit, bits[k], p.open_tile)
        assert amp_error(got, ref, p.n) < TOL["bf16x3"], k


def test_full_rotation_batch_small_members_vs_statevector(api):
    """The whole 256-circuit rotation batch of the benchmark (seed 0) in one
    bf16x3 qflex_amplitudes_grad call: the amplitude of every member of at
    most 20 qubits (85 of the 256) against the state vector, and every angle
    gradient of the 17 members of 16 qubits against the state-vector adjoint."""
    probs = rotation_batch(256, 0)
    bits = [random_bitstrings(p.n, 1, 5000 + i) for i, p in enumerate(probs)]
    flat_bits = torch.from_numpy(np.concatenate([b.reshape(-1) for b in bits])).cuda()
    flat_th = torch.from_numpy(np.concatenate([p.circuit.angles for p in probs])).cuda()
    multi = api.Plan(probs, "bf16x3", device=0)
    g = torch.zeros((1, len(probs), 2), dtype=torch.float64, device="cuda")
    g[..., 0] = 1.0
    amps, grad = multi.amplitudes_grad(flat_bits, flat_th, g)
    multi.sync()
    amps, grad = amps.cpu().numpy(), grad.cpu().numpy()
    lay = multi.layout(1)
    multi.close()
    small = [k for k, p in enumerate(probs) if p.n <= 20]
    assert len(small) == 85
    n_grad = 0
    for k in small:
        p = probs[k]
        ref = SV.amplitudes(p.circuit, bits[k], [])
        assert amp_error(amps[lay["amps"][k]:lay["amps"][k + 1]], ref, p.n) < TOL["bf16x3"], k
        if p.n == 16:
            gref = GR.statevector_adjoint(p.circuit, bits[k], [], np.ones((1, 1), dtype=np.complex128))
            gk = grad[lay["params"][k]:lay["params"][k + 1]]
            assert np.max(np.abs(gk - gref)) / (0.5 * np.sqrt(2.0 ** -p.n)) < 2e-4, k
            n_grad += 1
    assert n_grad == 17
