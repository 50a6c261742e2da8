"""GPU parity of the configurations the cut search finds when it may cut two
bonds whose CZ projector bits are tied (Methods, "Cutting indexes": a path
fixes the cut bonds; tied bits leave most paths identically zero), at the
bench's sizes: one path that does not vanish identically against the
oracle's contraction of the same path, a vanishing path against exact
zeros, and the FP64 norm of the path."""
import numpy as np
import pytest

from oracle import network as NW
from qflex_inputs import c2_problem, diamond_problem, random_bitstrings
from qflex_inputs.problems import Problem
from tests.gpu_util import amp_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# Both searched plans run more than 36 tensor-core products (40 on the 7x7
# grid, 45 on the 70-qubit diamond), where bf16 hi + lo operands measured
# 1.1e-4 to 1.2e-4; a bf16x3 plan of that length stores scaled fp16 planes
# instead (plane_format 3), and the split-precision bound of 1e-4 holds.
LONG_CHAIN_BF16X3 = 1e-4
# The search's result on these inputs, as the host tests pin it on x86-64
# (cuts, paths, nonzero paths): host code is built without FMA contraction,
# so the GB300's aarch64 host must find the same plan.
CASES = {
    "grid7x7_d32": (lambda: c2_problem(0), 24, 4, 32, LONG_CHAIN_BF16X3, ([32, 33, 80], 4096, 256)),
    "bris70_d32": (lambda: diamond_problem(32, 0), 28, 4, 8, LONG_CHAIN_BF16X3, ([100, 101, 72, 73], 65536, 256)),
}


@pytest.fixture(scope="module")
def api():
    from paper_1811_09599_gb300 import api
    api._lib.load(build_if_missing=True)
    return api


@pytest.mark.parametrize("case", sorted(CASES))
def test_searched_tied_cuts_path(api, case):
    make, log2_limit, max_new, trials, tol, pinned = CASES[case]
    base = make()
    r = api.search_ordering(Problem(base.circuit, [], base.open_tile, None), 1 << log2_limit, max_new,
                            trials=trials, seed=0)
    assert r["fits"] and (list(r["cuts"]), int(r["n_slices"]), int(r["n_nonzero_slices"])) == pinned
    prob = Problem(base.circuit, r["cuts"], base.open_tile, r["ordering"])
    nz = NW.nonzero_slices(prob.circuit, prob.cut_edges)
    assert len(nz) == r["n_nonzero_slices"]
    s = nz[int(np.random.default_rng(99).integers(len(nz)))]
    bs = random_bitstrings(prob.n, 1, 80)
    ref = NW.slice_amplitudes(prob, bs[0], s)
    plan = api.Plan(prob, "bf16x3", device=0)
    assert plan.info()["plane_format"] == 3          # long chain: scaled fp16 planes
    assert list(plan.nonzero_slices()) == nz
    b = torch.from_numpy(bs).cuda()
    got = plan.amplitudes(b, None, [s])
    plan.sync()
    nrm = api.norm(got).item()
    assert abs(nrm - float(np.sum(np.abs(ref) ** 2))) < 1e-3 * nrm
    # a kept path carries 1/len(nz) of the norm: the floor of the relative error
    assert amp_error(got.cpu().numpy(), ref, prob.n, 1.0 / len(nz)) < tol
    z = min(set(range(int(r["n_slices"]))) - set(nz))
    assert torch.count_nonzero(plan.amplitudes(b, None, [z])).item() == 0
    plan.close()
