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
