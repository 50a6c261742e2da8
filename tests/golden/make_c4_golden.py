"""Write tests/golden/c4_slices.json: the FP64 oracle's amplitudes of paths 0
and 1 of the 7x7 grid workload of depth 1+40+1 (bond dimension 32, two
region cuts = 1024 paths, 6-qubit open tile), one bitstring.

Methods, "Cutting indexes": a path fixes the values of the cut bonds and the
amplitude is the sum over them; SI A ("Contraction of RQCs on rectangular
grids") builds regions A (top left), B (top right), D (bottom right), takes
A.B, then (A.B).D, and absorbs region C (bottom left, holding the open tile)
qubit by qubit.  At bond dimension 32 each region tensor has 2^30 entries
(16 GiB in complex128), so the oracle cuts two more bonds itself, which the
same sum-over-paths identity allows:
  e1 = the A-C bond of column 0 (value v), which is contracted when C's
       qubit (r0, 0) is absorbed;
  e2 = the B-D bond of column J-2 (value w), which is contracted in (A.B).D.
Then every tensor has at most 2^25 entries and the sums are taken where the
bond closes:
  ABD_v = sum_w (A_v . B_w) . D_w;
  R     = sum_v (ABD_v with C's row r0 absorbed);
  amp   = R with the rest of C absorbed (the tile legs open, in tile order).
Every contraction is oracle.network.contract_pair (numpy.tensordot in
complex128) on oracle.network grid tensors; B_w and D_w are kept for all w,
A_v is built per v.  test_golden.py checks this function against
oracle.network.slice_amplitudes on the same lattice at small depths.

Calls only oracle/ (and the seeded input generators); no value comes from
the GPU path.  Run from the repository root (about 35 GB of host memory and
~1.5 h on 8 cores):

    python tests/golden/make_c4_golden.py
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import network as NW  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c4_slices.json")
CIRCUIT_SEED, BITSTRING_SEED, PATHS = 0, 2000, (0, 1)


def _chain(net, seq, log=None):
    """Absorb the tensors of `seq[1:]` into seq[0] in order (qubit ids)."""
    arr, legs = net[seq[0]]
    for q in seq[1:]:
        b, lb = net[q]
        arr, legs = NW.contract_pair(arr, legs, b, lb)
    return arr, legs


def _add(acc, arr, legs):
    if acc is None:
        return [arr.copy(), legs]
    assert acc[1] == legs, "partial results must carry the same legs"
    acc[0] += arr
    return acc


def region_split_amplitudes(prob, bits, s, r0=3, c0=3, log=print):
    """Amplitudes of path s of an I x J region problem (qflex_inputs
    grid_problem with cuts: right cut on the B-D edge of the last column,
    bottom cut on the C-D edge of the last row), computed with the two extra
    oracle cuts e1, e2 described in the module docstring."""
    circ = prob.circuit
    lat = circ.lattice
    rows = 1 + max(r for r, _ in lat.coords)
    cols = 1 + max(c for _, c in lat.coords)
    q = lat.qid
    tile = list(prob.open_tile)
    e1 = lat.edge_id((r0 - 1, 0), (r0, 0))
    e2 = lat.edge_id((r0 - 1, cols - 2), (r0, cols - 2))
    assert e1 not in prob.cut_edges and e2 not in prob.cut_edges
    K = NW.bond_exponents(circ)
    tensors = NW.all_grid_tensors(circ)
    vals = NW.slice_values(circ, prob.cut_edges, s)

    def fixed_net(extra):
        fx_bonds = {("e", e): v for e, v in vals.items()}
        fx_bonds.update({("e", e): v for e, v in extra.items()})
        net = {}
        for qq, (arr, legs) in enumerate(tensors):
            fx = dict(fx_bonds)
            if qq not in tile:
                fx[("o", qq)] = int(bits[qq])
            net[qq] = NW._fix(arr, legs, fx)
        return net

    A = [q(r, c) for c in range(c0) for r in range(r0)]
    B = [q(r, c) for c in range(cols - 1, c0 - 1, -1) for r in range(r0)]
    D = [q(r, c) for c in range(cols - 1, c0, -1) for r in range(rows - 1, r0 - 1, -1)]
    D += [q(r, c0) for r in range(rows - 1, r0 - 1, -1)]
    C_first = [q(r0, c) for c in range(c0 - 1, -1, -1)]          # closes e1
    C_rest = [q(r, c) for r in range(r0 + 1, rows) for c in range(c0 - 1, -1, -1)]
    n1, n2 = 1 << int(K[e1]), 1 << int(K[e2])
    t0 = time.time()
    Bw, Dw = [], []
    for w in range(n2):
        net = fixed_net({e2: w})
        Bw.append(_chain(net, B))
        Dw.append(_chain(net, D))
    if log:
        log(f"  B_w, D_w for {n2} values: {time.time() - t0:.0f} s")
    R = None
    for v in range(n1):
        Av = _chain(fixed_net({e1: v}), A)
        abd = None
        for w in range(n2):
            ab = NW.contract_pair(Av[0], Av[1], Bw[w][0], Bw[w][1])
            abd = _add(abd, *NW.contract_pair(ab[0], ab[1], Dw[w][0], Dw[w][1]))
        net = fixed_net({e1: v})
        arr, legs = abd
        for qq in C_first:
            arr, legs = NW.contract_pair(arr, legs, *net[qq])
        R = _add(R, arr, legs)
        if log:
            log(f"  v = {v + 1}/{n1}: {time.time() - t0:.0f} s")
    del Bw, Dw
    net = fixed_net({})
    arr, legs = R
    for qq in C_rest:
        arr, legs = NW.contract_pair(arr, legs, *net[qq])
    want = [("o", qq) for qq in tile]
    assert sorted(legs) == sorted(want)
    arr = np.transpose(arr, [legs.index(l) for l in want]) if want else arr
    return np.asarray(arr, dtype=np.complex128).reshape(-1)


def main() -> None:
    from qflex_inputs import c4_problem, random_bitstrings
    prob = c4_problem(CIRCUIT_SEED)
    bits = random_bitstrings(prob.n, 1, BITSTRING_SEED)[0]
    doc = {
        "what": "FP64 oracle amplitudes of paths 0 and 1 of the 7x7 depth 1+40+1 workload, one bitstring",
        "cite": "Methods 'Cutting indexes'; SI A 'Contraction of RQCs on rectangular grids' (7x7x(1+40+1))",
        "writer": "tests/golden/make_c4_golden.py (region_split_amplitudes: two extra oracle cuts, "
                  "oracle.network.contract_pair in complex128)",
        "problem": prob.name, "circuit_seed": CIRCUIT_SEED,
        "bitstrings": {"seed": BITSTRING_SEED, "count": 1, "index": 0},
        "bits": [int(x) for x in bits], "open_tile": [int(x) for x in prob.open_tile],
        "n_paths": int(NW.n_slices(prob.circuit, prob.cut_edges)), "paths": {},
        "cores": len(os.sched_getaffinity(0)),
    }
    for s in PATHS:
        t0 = time.time()
        print(f"path {s}", flush=True)
        amp = region_split_amplitudes(prob, bits, s, log=lambda m: print(m, flush=True))
        doc["paths"][str(s)] = {"re": [float(x) for x in amp.real], "im": [float(x) for x in amp.imag],
                                "seconds": round(time.time() - t0, 1)}
        with open(OUT, "w") as f:
            json.dump(doc, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
