"""Batch of uneven rotation circuits (4x4..6x6 grids, depth 1+16..32+1,
Rx/Ry/Rz with uniform random angles): amplitudes and gradients with respect
to every angle, checked on sampled members against the oracle."""
import numpy as np
import pytest

from oracle import gradients as GR
from oracle import network as NW
from oracle import statevector as SV
from qflex_inputs import random_bitstrings, rotation_batch
from tests.gpu_util import amp_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1811_09599_gb300 import api
    api._lib.load(build_if_missing=True)
    return api


BATCH = rotation_batch(256, 0)


def _pick(pred):
    return next(p for p in BATCH if pred(p))


def _run(api, prob, prec, seed):
    bs = random_bitstrings(prob.n, 1, seed)
    plan = api.Plan(prob, prec, device=0)
    g = np.array([[1.0 + 0.5j]])
    amps, grad = plan.amplitudes_grad(torch.from_numpy(bs).cuda(),
                                      torch.from_numpy(prob.circuit.angles).cuda(),
                                      torch.from_numpy(g).cuda())
    plan.sync()
    return bs, g, amps.cpu().numpy(), grad.cpu().numpy(), plan


def _gerr(got, ref, g, n):
    return float(np.max(np.abs(got - ref)) / (np.abs(g).max() * 0.5 * np.sqrt(2.0 ** -n)))


@pytest.mark.parametrize("shape", [(4, 4), (4, 5)])
def test_batch_member_vs_statevector_adjoint(api, shape):
    prob = _pick(lambda p: (p.circuit.lattice.name == f"grid{shape[0]}x{shape[1]}"))
    bs, g, amps, grad, _ = _run(api, prob, "fp32", 11)
    assert amp_error(amps, SV.amplitudes(prob.circuit, bs, []), prob.n) < 1e-5
    ref = GR.statevector_adjoint(prob.circuit, bs, [], g)
    assert _gerr(grad, ref, g, prob.n) < 2e-5


def test_batch_6x6_shift_rule_and_fd(api):
    """A 36-qubit member: sampled angles against the oracle's shift rule, and
    GPU central differences as an independent check."""
    prob = _pick(lambda p: p.circuit.lattice.name == "grid6x6" and p.circuit.depth <= 20)
    bs, g, amps, grad, plan = _run(api, prob, "fp32", 12)
    T = NW.all_grid_tensors(prob.circuit)
    ref_amp = NW.slice_amplitudes(prob, bs[0], 0, tensors=T)
    assert amp_error(amps, ref_amp, prob.n) < 1e-5
    params = [1, prob.circuit.n_params // 3, prob.circuit.n_params - 2]
    damp = GR.shift_rule(lambda th: NW.amplitudes(prob, bs, angles=th)[0], prob.circuit.angles, params)
    assert _gerr(grad[params], GR.loss_gradient(damp, g), g, prob.n) < 2e-5
    b = torch.from_numpy(bs).cuda()
    h = 1e-2
    fd = []
    for p in params:
        tp, tm = prob.circuit.angles.copy(), prob.circuit.angles.copy()
        tp[p] += h
        tm[p] -= h
        ap = plan.amplitudes(b, torch.from_numpy(tp).cuda()).cpu().numpy()
        am = plan.amplitudes(b, torch.from_numpy(tm).cuda()).cpu().numpy()
        fd.append(np.real(np.conj(g) * (ap - am) / (2 * h)).sum())
    assert _gerr(grad[params], np.array(fd), g, prob.n) < 2e-3


def test_batch_split_precision_members(api):
    """Members run in bf16x3 agree with the oracle at the split tolerance."""
    for name in ("grid5x6", "grid6x5"):
        prob = _pick(lambda p: p.circuit.lattice.name == name and p.circuit.depth <= 24)
        bs, g, amps, grad, _ = _run(api, prob, "bf16x3", 13)
        ref = NW.slice_amplitudes(prob, bs[0], 0)
        assert amp_error(amps, ref, prob.n) < 1e-4
        assert np.all(np.isfinite(grad))


def test_batch_concurrent_streams_match_sequential(api):
    """Independent circuits of the batch run concurrently on several streams
    (as bench.py times them) give exactly the sequential amplitudes, and the
    same gradients up to the order of their FP64 atomic accumulation (each
    angle's gradient is summed with atomicAdd over grid-tensor entries):
    each plan owns its workspace and status word."""
    members = BATCH[:12]
    g = torch.ones((1, 1), dtype=torch.complex128, device="cuda")
    inputs = [(torch.from_numpy(random_bitstrings(p.n, 1, 900 + i)).cuda(),
               torch.from_numpy(p.circuit.angles).cuda()) for i, p in enumerate(members)]
    seq = []
    for p, (b, th) in zip(members, inputs):
        plan = api.Plan(p, "bf16x3", device=0)
        a, gr = plan.amplitudes_grad(b, th, g)
        plan.sync()
        seq.append((a.cpu().numpy(), gr.cpu().numpy()))
        plan.close()
    plans = [api.Plan(p, "bf16x3", device=0) for p in members]
    for pl in plans:
        pl.enable_gradients()
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in range(4)]
    outs = []
    for j, pl in enumerate(plans):
        st = streams[j % 4]
        st.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(st):
            outs.append(pl.amplitudes_grad(inputs[j][0], inputs[j][1], g, stream=st))
    torch.cuda.synchronize()
    for pl, (a, gr), (sa, sg) in zip(plans, outs, seq):
        pl.sync()
        assert np.array_equal(a.cpu().numpy(), sa)
        gc = gr.cpu().numpy()
        assert np.max(np.abs(gc - sg)) <= 1e-12 * np.max(np.abs(sg)) + 1e-300
