"""GPU parity of the angle gradients (qflex_amplitudes_grad) with the oracle.

L = Re sum_j conj(g_j) amp_j for a random complex cotangent g; the GPU
gradient of L w.r.t. every rotation angle is compared with the oracle's
state-vector adjoint (all angles), with the exact shift rule on the oracle
contraction (sampled angles), with central finite differences of the GPU's
own amplitudes, and through torch.autograd (QFlexAmplitudes).
"""
import numpy as np
import pytest

from oracle import gradients as GR
from oracle import network as NW
from oracle import statevector as SV
from qflex_inputs import grid_problem, random_bitstrings

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GTOL = {"fp32": 2e-5, "tf32x3": 2e-4, "bf16x3": 2e-4, "fp16x3": 2e-4}


@pytest.fixture(scope="module")
def api():
    from paper_1811_09599_gb300 import api
    api._lib.load(build_if_missing=True)
    return api


def grad_error(got, ref, g, n_qubits):
    """max |dgrad| / (||g|| * sqrt(2^-n) / 2): gradient error relative to the
    typical size of a rotation derivative of a Porter-Thomas amplitude."""
    scale = np.linalg.norm(np.asarray(g).reshape(-1)) * 0.5 * np.sqrt(2.0 ** -n_qubits)
    return float(np.max(np.abs(np.asarray(got) - np.asarray(ref))) / scale)


def _cotangent(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex128)


def _gpu_grad(api, prob, prec, bs, g, slices=None):
    plan = api.Plan(prob, prec, device=0)
    b = torch.from_numpy(np.ascontiguousarray(bs)).cuda()
    th = torch.from_numpy(prob.circuit.angles).cuda()
    amps, grad = plan.amplitudes_grad(b, th, torch.from_numpy(g).cuda(), slices)
    plan.sync()
    return amps.cpu().numpy(), grad.cpu().numpy(), plan


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3", "fp16x3"])
def test_grad_vs_statevector_adjoint(api, prec):
    """3x4, 1+20+1 rotations, two cuts (all slices), 2-qubit tile, 2 bitstrings."""
    prob = grid_problem(3, 4, 20, 8, r0=2, c0=2, cuts=True, tile_rows=1, tile_cols=2, rotations=True)
    bs = random_bitstrings(prob.n, 2, 8)
    g = _cotangent((2, 4), 1)
    amps, grad, _ = _gpu_grad(api, prob, prec, bs, g)
    ref_amps = SV.amplitudes(prob.circuit, bs, prob.open_tile)
    ref = GR.statevector_adjoint(prob.circuit, bs, prob.open_tile, g)
    assert np.max(np.abs(amps - ref_amps)) / np.sqrt(2.0 ** -prob.n) < 1e-3
    assert grad.shape == (prob.circuit.n_params,)
    assert grad_error(grad, ref, g, prob.n) < GTOL[prec], grad_error(grad, ref, g, prob.n)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_grad_4x5_cut_vs_shift_rule_and_fd(api, prec):
    """4x5, 1+24+1 rotations (bonds 8), two cuts (64 slices), 4-qubit tile:
    sampled angles against the oracle's exact shift rule; GPU central
    differences of the GPU amplitudes as an independent check."""
    prob = grid_problem(4, 5, 24, 3, r0=2, c0=2, cuts=True, tile_rows=2, tile_cols=2, rotations=True)
    bs = random_bitstrings(prob.n, 1, 3)
    g = _cotangent((1, 16), 2)
    amps, grad, plan = _gpu_grad(api, prob, prec, bs, g)
    params = [0, 7, prob.circuit.n_params // 2, prob.circuit.n_params - 1]
    damp = GR.shift_rule(lambda th: NW.amplitudes(prob, bs, angles=th)[0], prob.circuit.angles, params)
    ref = GR.loss_gradient(damp, g)
    assert grad_error(grad[params], ref, g, prob.n) < GTOL[prec]
    if prec == "fp32":
        b = torch.from_numpy(bs).cuda()
        h = 1e-2
        fd = []
        for p in params:
            tp = prob.circuit.angles.copy()
            tm = tp.copy()
            tp[p] += h
            tm[p] -= h
            ap = plan.amplitudes(b, torch.from_numpy(tp).cuda()).cpu().numpy()
            am = plan.amplitudes(b, torch.from_numpy(tm).cuda()).cpu().numpy()
            fd.append(np.real(np.conj(g) * (ap - am) / (2 * h)).sum())
        assert grad_error(grad[params], np.array(fd), g, prob.n) < 2e-3


def test_autograd_function(api):
    """torch.autograd through QFlexAmplitudes gives the oracle gradient."""
    prob = grid_problem(3, 3, 16, 4, r0=1, c0=1, cuts=True, tile_rows=1, tile_cols=1, rotations=True)
    bs = random_bitstrings(prob.n, 3, 4)
    w = _cotangent((3, 2), 3)
    plan = api.Plan(prob, "fp32", device=0)
    th = torch.from_numpy(prob.circuit.angles).cuda().requires_grad_(True)
    amps = api.QFlexAmplitudes.apply(th, torch.from_numpy(bs).cuda(), plan)
    loss = (amps * torch.from_numpy(w).cuda().conj()).real.sum()
    loss.backward()
    ref = GR.statevector_adjoint(prob.circuit, bs, prob.open_tile, w)
    assert grad_error(th.grad.cpu().numpy(), ref, w, prob.n) < GTOL["fp32"]


def test_grad_partial_slices_and_plain_gates(api):
    """A fraction of the slices (the gradient of the partial sum), and gates
    without angles (plain RQC gates mixed in) contribute nothing spurious."""
    prob = grid_problem(3, 4, 16, 2, r0=2, c0=2, cuts=True, tile_rows=1, tile_cols=2, rotations=True)
    # turn half of the rotations back into fixed gates by dropping their angle
    for gate in prob.circuit.gates[::2]:
        if gate.kind in ("RX", "RY", "RZ"):
            gate.kind, gate.param = "H", -1
    bs = random_bitstrings(prob.n, 1, 2)
    g = _cotangent((1, 4), 4)
    sl = [0, 3, 9]
    _, grad, _ = _gpu_grad(api, prob, "fp32", bs, g, sl)
    used = sorted({gt.param for gt in prob.circuit.gates if gt.param >= 0})
    damp = GR.shift_rule(lambda th: NW.amplitudes(prob, bs, slices=sl, angles=th)[0],
                         prob.circuit.angles, used)
    ref = GR.loss_gradient(damp, g)
    assert grad_error(grad[used], ref, g, prob.n) < GTOL["fp32"]
    unused = sorted(set(range(prob.circuit.n_params)) - set(used))
    assert np.all(grad[unused] == 0)


@pytest.fixture(scope="module")
def oracle_6x6():
    """The 6x6 depth 1+32+1 rotation circuit, its bitstring and cotangent, and
    the oracle's amplitude and shift-rule loss gradient for sampled angles."""
    prob = grid_problem(6, 6, 32, 99, cuts=False, tile_rows=0, rotations=True)
    bs = random_bitstrings(prob.n, 1, 6)
    g = _cotangent((1, 1), 4)
    n = prob.circuit.n_params
    params = [0, n // 3, 2 * n // 3, n - 1]
    amp_fn = lambda th: NW.amplitudes(prob, bs, angles=th)[0]
    ref_amp = amp_fn(prob.circuit.angles)
    ref = GR.loss_gradient(GR.shift_rule(amp_fn, prob.circuit.angles, params), g)
    return prob, bs, g, params, ref_amp, ref


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_grad_6x6_long_reverse_products_vs_shift_rule(api, oracle_6x6, prec):
    """6x6, 1+32+1 rotations (bonds 16), no cuts, one amplitude: its reverse
    pass has products with few outputs and a long K (256 x 256 outputs over
    K = 65536 for the 65536 x 256 x 256 absorbs), which run split-K; sampled
    angles against the oracle's exact shift rule on its own contraction."""
    prob, bs, g, params, ref_amp, ref = oracle_6x6
    amps, grad, plan = _gpu_grad(api, prob, prec, bs, g)
    assert any((s["M"], s["N"], s["K"]) == (65536, 256, 256) for s in plan.steps(1))
    assert np.max(np.abs(amps.reshape(-1) - ref_amp)) / np.sqrt(2.0 ** -prob.n) < 1e-3
    assert grad_error(grad[params], ref, g, prob.n) < GTOL[prec], grad_error(grad[params], ref, g, prob.n)
