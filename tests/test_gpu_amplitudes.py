"""GPU parity of the whole path (qflex_amplitudes) against the FP64 oracle.

Small cases compare every amplitude with the state vector / oracle
contraction; the full-size 7x7 workloads compare sampled per-slice values
the oracle computes one by one.
"""
import numpy as np
import pytest

from oracle import network as NW
from oracle import selection as SEL
from oracle import statevector as SV
from qflex_inputs import (c1_problem, c2_problem, c4_problem, grid_problem, random_bitstrings)
from tests.gpu_util import TOL, amp_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = ["fp32", "tf32x3", "bf16x3", "fp16x3"]


@pytest.fixture(scope="module")
def api():
    from paper_1811_09599_gb300 import api
    api._lib.load(build_if_missing=True)
    return api


def _run(api, prob, prec, bs, slices=None, angles=None):
    plan = api.Plan(prob, prec, device=0)
    b = torch.from_numpy(np.ascontiguousarray(bs)).cuda()
    a = torch.from_numpy(np.asarray(angles, dtype=np.float64)).cuda() if angles is not None else None
    out = plan.amplitudes(b, a, slices).cpu().numpy()
    plan.sync()
    return out, plan


@pytest.mark.parametrize("prec", PRECS)
def test_c1_full_tile_vs_statevector(api, prec):
    """4x4, 1+16+1, no cuts, tile = all 16 qubits: 65,536 amplitudes vs the
    FP64 state vector, and the FP64 norm on the GPU equals 1."""
    prob = c1_problem(0, full_tile=True)
    bs = random_bitstrings(16, 1, 0)
    got, plan = _run(api, prob, prec, bs)
    ref = SV.final_state(prob.circuit).reshape(1, -1)
    assert amp_error(got, ref, 16) < TOL[prec]
    nrm = api.norm(torch.from_numpy(got).cuda()).item()
    assert abs(nrm - 1.0) < 10 * TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_c1_sixteen_bitstrings(api, prec):
    prob = c1_problem(3, full_tile=False)
    bs = random_bitstrings(16, 16, 3)
    got, _ = _run(api, prob, prec, bs)
    ref = SV.amplitudes(prob.circuit, bs, [])
    assert amp_error(got, ref, 16) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_cut_grid_all_and_partial_slices(api, prec):
    """4x5, 1+24+1 (bonds 8), two cuts (64 slices), 4-qubit tile: full sum vs
    state vector; every single slice vs the oracle's slice; a fraction-f sum."""
    prob = grid_problem(4, 5, 24, 5, r0=2, c0=2, cuts=True, tile_rows=2, tile_cols=2)
    bs = random_bitstrings(prob.n, 3, 5)
    P = NW.n_slices(prob.circuit, prob.cut_edges)
    assert P == 64
    got, plan = _run(api, prob, prec, bs)
    ref = SV.amplitudes(prob.circuit, bs, prob.open_tile)
    assert amp_error(got, ref, prob.n) < TOL[prec]
    tensors = NW.all_grid_tensors(prob.circuit)
    for s in (0, 17, 63):
        g1 = plan.amplitudes(torch.from_numpy(bs[:1]).cuda(), None, [s]).cpu().numpy()
        r1 = NW.slice_amplitudes(prob, bs[0], s, tensors=tensors)
        assert amp_error(g1, r1, prob.n, 1.0 / P) < TOL[prec]
    sel = SEL.select_slices(P, 0.25, 11)
    assert list(plan.select_slices(0.25, 11)) == sel
    gf = plan.amplitudes(torch.from_numpy(bs).cuda(), None, sel).cpu().numpy()
    rf = NW.amplitudes(prob, bs, sel)
    assert amp_error(gf, rf, prob.n, len(sel) / P) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_rotation_circuit_with_angles(api, prec):
    prob = grid_problem(3, 4, 20, 8, r0=2, c0=2, cuts=True, tile_rows=1, tile_cols=2,
                        rotations=True)
    bs = random_bitstrings(prob.n, 2, 8)
    got, _ = _run(api, prob, prec, bs, angles=prob.circuit.angles)
    ref = SV.amplitudes(prob.circuit, bs, prob.open_tile)
    assert amp_error(got, ref, prob.n) < TOL[prec]


def test_vanishing_paths_skipped(api):
    """3x4, 1+20+1 rotations, two cuts: R_Z between CZ projector halves makes
    half the paths vanish identically.  The sum over all paths, which skips
    them, equals the sum over the oracle's list of the others bit for bit
    (the same kernels run), a list of vanishing paths gives exact zeros,
    and the total matches the state vector."""
    prob = grid_problem(3, 4, 20, 8, r0=2, c0=2, cuts=True, tile_rows=1, tile_cols=2, rotations=True)
    nz = NW.nonzero_slices(prob.circuit, prob.cut_edges)
    P = NW.n_slices(prob.circuit, prob.cut_edges)
    zero = sorted(set(range(P)) - set(nz))
    assert len(zero) > 0
    bs = random_bitstrings(prob.n, 2, 12)
    plan = api.Plan(prob, "bf16x3", device=0)
    b = torch.from_numpy(bs).cuda()
    th = torch.from_numpy(prob.circuit.angles).cuda()
    assert list(plan.nonzero_slices()) == nz
    full = plan.amplitudes(b, th)
    part = plan.amplitudes(b, th, nz)
    assert torch.equal(full, part)
    assert torch.count_nonzero(plan.amplitudes(b, th, zero)).item() == 0
    assert np.max(np.abs(NW.amplitudes(prob, bs, zero))) == 0.0
    ref = SV.amplitudes(prob.circuit, bs, prob.open_tile)
    assert amp_error(full.cpu().numpy(), ref, prob.n) < TOL["bf16x3"]
    plan.sync()


def test_slice_order_and_repeats_are_consistent(api):
    """Slice lists in any order give the same sum (memoised reuse must not
    leak values across bitstrings or slice orders)."""
    prob = grid_problem(4, 5, 24, 6, r0=2, c0=2, cuts=True, tile_rows=1, tile_cols=2)
    bs = random_bitstrings(prob.n, 2, 6)
    plan = api.Plan(prob, "fp32", device=0)
    b = torch.from_numpy(bs).cuda()
    a = plan.amplitudes(b, None, list(range(64))).cpu().numpy()
    rng = np.random.default_rng(0)
    c = plan.amplitudes(b, None, list(rng.permutation(64))).cpu().numpy()
    assert np.max(np.abs(a - c)) <= 1e-6 * np.max(np.abs(a))


def test_empty_batch_and_bad_slice(api):
    prob = grid_problem(3, 3, 8, 1, r0=1, c0=1, cuts=False, tile_rows=1, tile_cols=1)
    plan = api.Plan(prob, "fp32", device=0)
    out = plan.amplitudes(torch.zeros((0, 9), dtype=torch.uint8, device="cuda"))
    assert out.shape == (0, 2)
    with pytest.raises(api._lib.QFlexError):
        plan.amplitudes(torch.zeros((1, 9), dtype=torch.uint8, device="cuda"), None, [1])


_C2_REF = {}


def _c2_reference(prob, bits, s):
    if s not in _C2_REF:
        if "tensors" not in _C2_REF:
            _C2_REF["tensors"] = NW.all_grid_tensors(prob.circuit)
        _C2_REF[s] = NW.slice_amplitudes(prob, bits, s, tensors=_C2_REF["tensors"])
    return _C2_REF[s]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "fp32", "fp16x3"])
def test_c2_full_size_sampled_slices(api, prec):
    """7x7, 1+32+1, two cuts (256 slices), 6-qubit tile: two sampled slices of
    one bitstring vs the oracle's slice contraction (full-size launch shapes:
    2^12 x 2^12 x 2^12 GEMMs, 2^24-entry permutations)."""
    prob = c2_problem(0)
    bs = random_bitstrings(prob.n, 1, 1234)
    plan = api.Plan(prob, prec, device=0)
    b = torch.from_numpy(bs).cuda()
    for s in (5, 200):
        got = plan.amplitudes(b, None, [s]).cpu().numpy()
        ref = _c2_reference(prob, bs[0], s)
        assert amp_error(got, ref, prob.n, 1.0 / 256) < TOL[prec], s
    plan.sync()


def test_c4_full_size_split_vs_fp32(api):
    """7x7, 1+40+1 (bond dimension 32, 2^15 x 2^15 x 2^15 GEMMs, 2^30-entry
    tensors), slice 0 of one bitstring: bf16x3 against the FP32 path (the FP64
    oracle cannot contract a slice of this size in test time; the 2^15-long
    GEMM accuracy itself is pinned against complex128 in test_gpu_kernels)."""
    prob = c4_problem(0)
    bs = torch.from_numpy(random_bitstrings(prob.n, 1, 2000)).cuda()
    res = {}
    for prec in ("bf16x3", "fp32"):
        plan = api.Plan(prob, prec, device=0)
        res[prec] = plan.amplitudes(bs, None, [0]).cpu().numpy()
        plan.sync()
        plan.close()
        torch.cuda.empty_cache()
    assert np.all(np.isfinite(res["fp32"])) and np.max(np.abs(res["fp32"])) > 0
    assert amp_error(res["bf16x3"], res["fp32"], prob.n, 1.0 / 1024) < TOL["bf16x3"]


def test_cuda_graph_replay(api):
    """qflex_plan_use_graphs: repeated calls replay a captured graph; changing
    the contents (not the address) of the bitstring buffer is seen by the
    replay; results equal the direct launches."""
    prob = grid_problem(4, 5, 24, 5, r0=2, c0=2, cuts=True, tile_rows=2, tile_cols=2)
    bs = random_bitstrings(prob.n, 3, 5)
    direct = api.Plan(prob, "bf16x3", device=0)
    ref = direct.amplitudes(torch.from_numpy(bs).cuda()).cpu().numpy()
    plan = api.Plan(prob, "bf16x3", device=0)
    plan.use_graphs(True)
    stream = torch.cuda.Stream()
    b = torch.from_numpy(bs).cuda()
    out = torch.empty((3, 16, 2), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(3):                      # direct, capture, replay
            got = plan.amplitudes(b, None, None, out=out, stream=stream)
        stream.synchronize()
        assert np.max(np.abs(got.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref)) + 1e-30
        bs2 = random_bitstrings(prob.n, 3, 99)
        b.copy_(torch.from_numpy(bs2))
        got2 = plan.amplitudes(b, None, None, out=out, stream=stream).cpu().numpy()
        stream.synchronize()
    ref2 = direct.amplitudes(torch.from_numpy(bs2).cuda()).cpu().numpy()
    assert np.max(np.abs(got2 - ref2)) <= 1e-12 * np.max(np.abs(ref2)) + 1e-30
    plan.sync()


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_autotune_keeps_results(api, prec):
    """qflex_plan_autotune only changes kernel configurations (tile width of
    the tensor-core GEMM, thin or tiled FP32 kernel for narrow steps).  The
    FP32 kernels sum in different orders, so the tuned path is not bitwise
    equal to the untuned one: a one-ulp change of an FP32 operand re-draws
    the low bits a bf16 hi/lo split drops, so the split error is re-drawn
    too.  Both runs must stay within the precision's tolerance of the oracle,
    and repeated tuned runs must be bitwise reproducible."""
    prob = c2_problem(0)
    bits = random_bitstrings(prob.n, 1, 1234)
    bs = torch.from_numpy(bits).cuda()
    plan = api.Plan(prob, prec, device=0)
    before = plan.amplitudes(bs, None, [5]).cpu().numpy()
    info = plan.autotune(2)
    assert info["shapes"] > 0 and info["gain_ms"] >= 0.0
    after = plan.amplitudes(bs, None, [5]).cpu().numpy()
    again = plan.amplitudes(bs, None, [5]).cpu().numpy()
    ref = _c2_reference(prob, bits[0], 5)
    assert amp_error(before, ref, prob.n, 1.0 / 256) < TOL[prec]
    assert amp_error(after, ref, prob.n, 1.0 / 256) < TOL[prec]
    assert np.array_equal(after, again)
    plan.sync()
