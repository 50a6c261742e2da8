"""Epilogue fusion: a tensor-core step writing its consumer's 3M operand
planes directly (bit-permuted into the consumer's layout) computes exactly
what the unfused path computes -- complex64 output, then a permutation that
splits it into the same planes.  Gradient calls run the forward unfused (the
reverse pass needs the complex64 intermediates), so their amplitudes must be
bit-identical to those of a plain call on the same plan."""
import numpy as np
import pytest

from oracle import network as NW
from qflex_inputs import grid_problem, random_bitstrings
from tests.gpu_util import TOL, amp_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1811_09599_gb300 import api
    api._lib.load(build_if_missing=True)
    return api


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "bf16", "tf32"])
def test_fused_equals_unfused_bitwise(api, prec):
    """5x5, 1+32+1 rotations (bond dimension 16), two cuts (256 slices),
    4-qubit tile, 2 bitstrings: 7 fused steps."""
    prob = grid_problem(5, 5, 32, 3, r0=2, c0=2, cuts=True, tile_rows=2, tile_cols=2, rotations=True)
    bs = torch.from_numpy(random_bitstrings(prob.n, 2, 3)).cuda()
    th = torch.from_numpy(prob.circuit.angles).cuda()
    plan = api.Plan(prob, prec, device=0)
    steps = plan.steps(2)
    assert any(s["out_fused"] for s in steps), "no fused step in this plan"
    fused = plan.amplitudes(bs, th).cpu().numpy()
    g = torch.ones((2, 16), dtype=torch.complex128, device="cuda")
    unfused, _ = plan.amplitudes_grad(bs, th, g)
    plan.sync()
    assert np.array_equal(fused, unfused.cpu().numpy())
    if prec in TOL:        # sampled slices against the oracle's slice contraction
        bits = random_bitstrings(prob.n, 2, 3)
        tensors = NW.all_grid_tensors(prob.circuit)
        for sl in (7, 200):
            got = plan.amplitudes(bs, th, [sl]).cpu().numpy()
            ref = np.stack([NW.slice_amplitudes(prob, b, sl, tensors=tensors) for b in bits])
            assert amp_error(got, ref, prob.n, 1.0 / 256) < TOL[prec], sl


def test_fused_plan_counts(api):
    """The 7x7 depth 1+32+1 plan fuses the absorb chains and both operands
    of the 4096^3 products: permutation traffic per bitstring falls by >2/3."""
    from qflex_inputs import c2_problem
    p = api.Plan(c2_problem(0), "bf16x3", device=-1)
    steps = p.steps(1)
    big = [s for s in steps if (s["M"], s["N"], s["K"]) == (4096, 4096, 4096)]
    assert all(s["a_fused"] and s["b_fused"] for s in big)
    fp32 = api.Plan(c2_problem(0), "fp32", device=-1)
    assert p.cost(1)["permute_bytes"] < fp32.cost(1)["permute_bytes"] / 3
    assert not any(s["out_fused"] or s["a_fused"] for s in fp32.steps(1))


def test_fused_fp16_planes_vs_oracle(api):
    """fp16x3 with fused planes: the producer scales its output by a power of
    two taken from the bound 3 K max|A| max|B| of its entries (known before
    the first entry is written), not from their measured maximum, so the
    planes differ from the unfused path's (gradient calls) in their scale but
    both sum to the oracle's amplitudes within the split tolerance."""
    prob = grid_problem(5, 5, 32, 3, r0=2, c0=2, cuts=True, tile_rows=2, tile_cols=2, rotations=True)
    bits = random_bitstrings(prob.n, 2, 3)
    bs = torch.from_numpy(bits).cuda()
    th = torch.from_numpy(prob.circuit.angles).cuda()
    plan = api.Plan(prob, "fp16x3", device=0)
    steps = plan.steps(2)
    assert sum(bool(s["out_fused"]) for s in steps) >= 5
    fused = plan.amplitudes(bs, th).cpu().numpy()
    g = torch.ones((2, 16), dtype=torch.complex128, device="cuda")
    unfused, _ = plan.amplitudes_grad(bs, th, g)
    plan.sync()
    assert amp_error(fused, unfused.cpu().numpy(), prob.n) < TOL["fp16x3"]
    tensors = NW.all_grid_tensors(prob.circuit)
    for sl in (7, 200):
        got = plan.amplitudes(bs, th, [sl]).cpu().numpy()
        plan.sync()
        ref = np.stack([NW.slice_amplitudes(prob, b, sl, tensors=tensors) for b in bits])
        assert amp_error(got, ref, prob.n, 1.0 / 256) < TOL["fp16x3"], sl


def test_profile_by_shape(api):
    """Profiled launches by product shape add up to the per-class totals, and
    every recorded shape is a product of the plan's schedule (the records the
    bench's per-shape roofline is computed from)."""
    prob = grid_problem(5, 5, 32, 3, r0=2, c0=2, cuts=True, tile_rows=2, tile_cols=2, rotations=True)
    bs = torch.from_numpy(random_bitstrings(prob.n, 2, 3)).cuda()
    th = torch.from_numpy(prob.circuit.angles).cuda()
    plan = api.Plan(prob, "bf16x3", device=0)
    plan.amplitudes(bs, th)
    plan.profile_start(["gemm_fp32", "gemm_tc"])
    plan.amplitudes(bs, th)
    tot = plan.profile_stop()
    shapes = plan.profile_shapes()
    plan.sync()
    sched = {(s["M"], s["N"], s["K"], s["kernel"] == "tensor_cores") for s in plan.steps(2)}
    for cls in ("gemm_fp32", "gemm_tc"):
        rows = [r for r in shapes if r["cls"] == cls]
        assert sum(r["launches"] for r in rows) == tot[cls]["launches"]
        assert np.isclose(sum(r["ms"] for r in rows), tot[cls]["ms"], rtol=1e-9, atol=1e-9)
        assert np.isclose(sum(r["mma_flops"] for r in rows), tot[cls]["mma_flops"], rtol=1e-12)
        for r in rows:
            assert (r["M"], r["N"], r["K"], cls == "gemm_tc") in sched, r
    assert tot["gemm_tc"]["launches"] > 0 and any(r["out_planes"] for r in shapes)
