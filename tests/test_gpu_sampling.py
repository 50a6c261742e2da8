"""Frugal rejection sampling on the GPU (qflex_frugal_sample) against the
oracle's restatement of the same procedure: identical accepted indices, and
the acceptance rates the paper prints (Methods, "Fast sampling technique")."""
import numpy as np
import pytest

from oracle import selection as SEL
from oracle import statevector as SV
from qflex_inputs import grid_problem, random_bitstrings

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1811_09599_gb300 import api
    api._lib.load(build_if_missing=True)
    return api


def _pt(nb, nc, n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((nb, nc)) + 1j * rng.standard_normal((nb, nc))) * np.sqrt(0.5 * 2.0 ** -n)


def test_frugal_bit_exact_vs_oracle(api):
    n = 24
    for nb, nc, M, seed in ((500, 30, 10.0, 1), (300, 64, 15.0, 2), (50, 4096, 10.0, 3), (7, 1, 10.0, 4)):
        amps = _pt(nb, nc, n, seed)
        got = api.frugal_sample(torch.from_numpy(amps).cuda(), n, M, seed).cpu().numpy()
        assert np.array_equal(got, SEL.frugal_sample(amps, n, M, seed)), (nb, nc)


def test_frugal_acceptance_rates(api):
    """95.76% (M=10, N_C=30) and 99.82% (N_C=60) from the paper."""
    n = 30
    for nc, want in ((30, 0.9576), (60, 0.9982)):
        amps = _pt(100000, nc, n, nc)
        acc = api.frugal_sample(torch.from_numpy(amps).cuda(), n, 10.0, 9).cpu().numpy()
        assert abs(np.mean(acc >= 0) - want) < 3e-3


def test_frugal_on_circuit_batches(api):
    """Batches = the open-tile amplitudes of several bitstrings of a circuit,
    computed by the GPU path; decisions equal the oracle's on the same
    amplitudes, and samples from the exact distribution have <pN> > 1."""
    prob = grid_problem(4, 5, 24, 5, r0=2, c0=2, cuts=True, tile_rows=2, tile_cols=3)
    bs = random_bitstrings(prob.n, 64, 5)
    plan = api.Plan(prob, "fp32", device=0)
    amps = plan.amplitudes(torch.from_numpy(bs).cuda())
    acc = api.frugal_sample(amps, prob.n, 10.0, 77).cpu().numpy()
    assert np.array_equal(acc, SEL.frugal_sample(amps.cpu().numpy(), prob.n, 10.0, 77))
    ref = SV.amplitudes(prob.circuit, bs, prob.open_tile)
    rows = np.nonzero(acc >= 0)[0]
    pN = np.abs(ref[rows, acc[rows]]) ** 2 * 2.0 ** prob.n
    assert len(rows) > 40 and pN.mean() > 1.2


# ------------------------------------------------------------ fidelity-f samples
def _mix_inputs(nb, n, seed):
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2, size=(nb, n), dtype=np.uint8)
    acc = rng.integers(-1, 256, size=nb).astype(np.int32)
    acc[rng.random(nb) < 0.2] = -1
    return bits, acc


@pytest.mark.parametrize("f", [0.0, 0.37, 1.0])
def test_fidelity_samples_bit_exact_vs_oracle(api, f):
    """Methods, "Fraction of perfect fidelity amplitudes": every sample, its
    source and the exact count equal the oracle's (integer work: bit-exact).
    70 qubits (two 64-bit draws per uniform sample), 8-qubit tile, more
    samples than one 1024-thread scan chunk and a ragged last chunk."""
    n, nb, ns = 70, 30000, 20000 + 317
    tile = [9, 3, 40, 41, 63, 64, 65, 69]
    bits, acc = _mix_inputs(nb, n, 5)
    s, src, k = api.fidelity_samples(torch.from_numpy(bits).cuda(), torch.from_numpy(acc).cuda(),
                                     tile, f, ns, seed=123)
    rs, rsrc, rk = SEL.fidelity_samples(bits, acc, tile, f, 123, ns)
    assert k == rk
    assert np.array_equal(src.cpu().numpy(), rsrc)
    assert np.array_equal(s.cpu().numpy(), rs)


def test_fidelity_samples_short_pool_and_edges(api):
    """More exact draws than accepted batches: QFLEX_ERR_ARG, and the draws
    past the pool are marked -2 with zero bits, as in the oracle; zero
    batches at f = 0 is fine; zero draws return at once."""
    import ctypes as C
    from paper_1811_09599_gb300 import QFlexError, _lib
    n, nb, ns = 12, 40, 200
    tile = [0, 5]
    bits, acc = _mix_inputs(nb, n, 8)
    bb, aa = torch.from_numpy(bits).cuda(), torch.from_numpy(acc).cuda()
    with pytest.raises(QFlexError, match="ARG"):
        api.fidelity_samples(bb, aa, tile, 1.0, ns, seed=4)
    lib = _lib.load()
    out = torch.empty((ns, n), dtype=torch.uint8, device="cuda")
    src = torch.empty(ns, dtype=torch.int32, device="cuda")
    k = C.c_int64()
    t = (C.c_int32 * 2)(*tile)
    st = lib.qflex_fidelity_samples(C.c_void_p(bb.data_ptr()), C.c_void_p(aa.data_ptr()), nb, t, 2, n, 1.0,
                                    C.c_uint64(4), ns, C.c_void_p(out.data_ptr()), C.c_void_p(src.data_ptr()),
                                    C.byref(k), None)
    assert st == 1 and k.value == ns
    rs, rsrc, rk = SEL.fidelity_samples(bits, acc, tile, 1.0, 4, ns)
    assert np.array_equal(src.cpu().numpy(), rsrc) and np.array_equal(out.cpu().numpy(), rs)
    assert np.sum(rsrc == -2) == ns - np.sum(acc >= 0)
    empty_b = torch.empty((0, n), dtype=torch.uint8, device="cuda")
    empty_a = torch.empty(0, dtype=torch.int32, device="cuda")
    s0, src0, k0 = api.fidelity_samples(empty_b, empty_a, tile, 0.0, 50, seed=4)
    assert k0 == 0 and np.all(src0.cpu().numpy() == -1)
    s1, _, k1 = api.fidelity_samples(bb, aa, tile, 0.5, 0, seed=4)
    assert k1 == 0 and s1.shape == (0, n)


@pytest.mark.parametrize("f", [0.3, 0.7])
def test_fidelity_sampling_pipeline_xeb(api, f):
    """The whole sampler on the GPU: open-tile amplitudes of a 16-qubit RQC
    for random bitstrings (qflex_amplitudes), frugal rejection per batch,
    then the fidelity-f mixture; the linear XEB of the samples against the
    oracle's exact probabilities is f (N sum p^2 - 1) within statistics."""
    prob = grid_problem(4, 4, 16, 6, r0=2, c0=3, cuts=False, tile_rows=2, tile_cols=3)
    n = prob.n
    nb, ns = 6000, 6000
    bits = random_bitstrings(n, nb, 44)
    plan = api.Plan(prob, "bf16x3", device=0)
    bb = torch.from_numpy(bits).cuda()
    amps = plan.amplitudes(bb)
    acc = api.frugal_sample(amps.reshape(nb, -1), n, 10.0, seed=3)
    s, src, k = api.fidelity_samples(bb, acc, prob.open_tile, f, ns, seed=17)
    plan.sync()
    psi = SV.final_state(prob.circuit).reshape(-1)
    p = np.abs(psi) ** 2
    idx = s.cpu().numpy().astype(np.int64) @ (1 << np.arange(n - 1, -1, -1))
    ideal = (2.0 ** n) * np.sum(p ** 2) - 1.0
    xeb = SEL.linear_xeb(p[idx], n)
    assert abs(k / ns - f) < 5 * np.sqrt(f * (1 - f) / ns)
    assert abs(xeb - f * ideal) < 5 * np.sqrt(2.0 / ns) + 0.05 * ideal, (xeb, f * ideal)
