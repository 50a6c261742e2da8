"""Full-size parity against stored FP64 oracle values (tests/golden/):

* the 7x7 depth 1+32+1 workload of the bench: one bitstring, all 256 paths
  summed (Methods "Cutting indexes"), 64 open-tile amplitudes; and the
  fraction of it over paths 0..15 (one value of the first cut);
* the 7x7 depth 1+40+1 workload (bond dimension 32, 1024 paths): paths 0
  and 1 of one bitstring, 64 amplitudes each (SI A's 7x7x(1+40+1) case).

The stored values were written by tests/golden/make_c2_fullsum.py and
make_c4_golden.py, which call only oracle/."""
import json
import os

import numpy as np
import pytest

from qflex_inputs import c2_problem, c4_problem, random_bitstrings
from tests.gpu_util import TOL, amp_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def api():
    from paper_1811_09599_gb300 import api
    api._lib.load(build_if_missing=True)
    return api


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _bits(doc, prob):
    b = random_bitstrings(prob.n, doc["bitstrings"]["count"], doc["bitstrings"]["seed"])[doc["bitstrings"]["index"]]
    assert [int(x) for x in b] == doc["bits"] and list(prob.open_tile) == doc["open_tile"]
    return torch.from_numpy(b[None, :].copy()).cuda()


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3", "tf32x3", "fp32"])
def test_c2_all_paths_vs_oracle(api, prec):
    doc = _load("c2_fullsum.json")
    prob = c2_problem(doc["circuit_seed"])
    assert prob.name == doc["problem"]
    b = _bits(doc, prob)
    plan = api.Plan(prob, prec, device=0)
    plan.autotune(2)
    full = plan.amplitudes(b).cpu().numpy().reshape(-1)
    part = plan.amplitudes(b, None, list(range(doc["partial_paths"]))).cpu().numpy().reshape(-1)
    plan.sync()
    ref_full = np.array(doc["full_re"]) + 1j * np.array(doc["full_im"])
    ref_part = np.array(doc["partial_re"]) + 1j * np.array(doc["partial_im"])
    assert amp_error(full, ref_full, prob.n) < TOL[prec]
    assert amp_error(part, ref_part, prob.n, doc["partial_paths"] / doc["n_paths"]) < TOL[prec]


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3", "tf32x3", "fp32"])
def test_c4_two_paths_vs_oracle(api, prec):
    doc = _load("c4_slices.json")
    prob = c4_problem(doc["circuit_seed"])
    assert prob.name == doc["problem"]
    b = _bits(doc, prob)
    plan = api.Plan(prob, prec, device=0)
    for s, ref in sorted(doc["paths"].items()):
        got = plan.amplitudes(b, None, [int(s)]).cpu().numpy().reshape(-1)
        plan.sync()
        r = np.array(ref["re"]) + 1j * np.array(ref["im"])
        assert amp_error(got, r, prob.n, 1.0 / doc["n_paths"]) < TOL[prec], s
    plan.close()
