"""Small single-purpose workloads for kernel profiling (ncu) of the hot path.

    python profile_cases.py <case>          (from the repository root)

Each case runs its kernel three times on cuda:0 (so `ncu -s 1 -c 1` captures
a warm launch) and prints "<case> ok".  Cases:
  perm    k_permute_tiled: random binary-axis permutation of 2^26 complex64
  thin    k_cgemm_thin: M=2^20, N=16, K=16 (the per-slice absorb of a grid
          tensor sharing one bond)
  tc      k_cgemm_tc bf16x3: M=N=K=4096 (the AB / ABD contraction of the
          7x7 grid at bond dimension 16)
  tcabs   k_cgemm_tc bf16x3: M=2^16, N=K=256 (a region absorb of one qubit)
  path    the 7x7 depth 1+32+1 workload for one bitstring and one right-cut
          value (slices 0..15, 1/16 of one bitstring with the same mix of
          launches as a full bench step)
  searched  the same workload planned by the cut search (tied cut pairs;
          2^24-entry limit, up to four new cuts, 32 passes): one bitstring,
          the first 16 nonzero paths
"""
from __future__ import annotations

import sys

import os

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from paper_1811_09599_gb300 import api  # noqa: E402


def main(case: str) -> None:
    api._lib.load(build_if_missing=True)
    torch.manual_seed(0)
    if case == "perm":
        m = 26
        x = torch.randn(1 << m, dtype=torch.complex64, device="cuda").view((2,) * m)
        perm = list(np.random.default_rng(7).permutation(m))
        for _ in range(3):
            api.permute(x, perm)
    elif case == "thin":
        a = torch.randn(1 << 20, 16, dtype=torch.complex64, device="cuda")
        b = torch.randn(16, 16, dtype=torch.complex64, device="cuda")
        for _ in range(3):
            api.cgemm(a, b, "fp32")
    elif case in ("tc", "tcabs"):
        M, N, K = (4096, 4096, 4096) if case == "tc" else (1 << 16, 256, 256)
        a = torch.randn(M, K, dtype=torch.complex64, device="cuda")
        b = torch.randn(N, K, dtype=torch.complex64, device="cuda")
        for _ in range(3):
            api.cgemm(a, b, "bf16x3")
    elif case == "path":
        from qflex_inputs import c2_problem, random_bitstrings
        prob = c2_problem(0)
        plan = api.Plan(prob, "bf16x3", device=0)
        bits = torch.from_numpy(random_bitstrings(prob.n, 1, 1000)).cuda()
        for _ in range(3):
            plan.amplitudes(bits, None, list(range(16)))
        plan.sync()
    elif case == "searched":
        from qflex_inputs import c2_problem, random_bitstrings
        from qflex_inputs.problems import Problem
        base = c2_problem(0)
        r = api.search_ordering(Problem(base.circuit, [], base.open_tile, None), 1 << 24, 4, trials=32, seed=0)
        plan = api.Plan(Problem(base.circuit, r["cuts"], base.open_tile, r["ordering"]), "bf16x3", device=0)
        bits = torch.from_numpy(random_bitstrings(base.n, 1, 1000)).cuda()
        paths = list(plan.nonzero_slices()[:16])
        for _ in range(3):
            plan.amplitudes(bits, None, paths)
        plan.sync()
    else:
        raise SystemExit(f"unknown case {case}")
    torch.cuda.synchronize()
    print(case, "ok")


if __name__ == "__main__":
    main(sys.argv[1])
