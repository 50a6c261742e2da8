"""Write tests/golden/c2_fullsum.json: the FP64 oracle's amplitudes of one
bitstring of the 7x7 grid workload (depth 1+32+1, two region cuts = 256
paths, 6-qubit open tile) summed over every path.

Methods, "Cutting indexes": the amplitude is the sum over all values of the
cut bonds; each path is contracted here by oracle.network.slice_amplitudes
(plain tensordot along the region ordering of SI A), accumulated in
ascending path order in complex128.  The file also keeps the partial sum
over paths 0..15 (one value of the first, "right", cut), so that a shorter
GPU test can compare a fraction-f sum.

Calls only oracle/ (and the seeded input generators); no value comes from
the GPU path.  Run from the repository root:

    python tests/golden/make_c2_fullsum.py            # ~40 min on 8 cores
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import network as NW  # noqa: E402
from qflex_inputs import c2_problem, random_bitstrings  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_fullsum.json")
CIRCUIT_SEED, BITSTRING_SEED, BITSTRING_INDEX, N_BITSTRINGS = 0, 1000, 0, 8
PARTIAL = 16


def main() -> None:
    prob = c2_problem(CIRCUIT_SEED)
    bits = random_bitstrings(prob.n, N_BITSTRINGS, BITSTRING_SEED)[BITSTRING_INDEX]
    tensors = NW.all_grid_tensors(prob.circuit)
    P = NW.n_slices(prob.circuit, prob.cut_edges)
    total = np.zeros(1 << len(prob.open_tile), dtype=np.complex128)
    partial = None
    t0 = time.time()
    for s in range(P):
        total += NW.slice_amplitudes(prob, bits, s, tensors=tensors)
        if s + 1 == PARTIAL:
            partial = total.copy()
        print(f"path {s + 1}/{P}  {time.time() - t0:.0f} s", flush=True)
    doc = {
        "what": "FP64 oracle amplitudes of one bitstring of the 7x7 grid workload, summed over all paths",
        "cite": "Methods 'Cutting indexes' (sum over paths); SI A 'Contraction of RQCs on rectangular grids'",
        "writer": "tests/golden/make_c2_fullsum.py (oracle.network.slice_amplitudes, ascending path order)",
        "problem": prob.name, "circuit_seed": CIRCUIT_SEED,
        "bitstrings": {"seed": BITSTRING_SEED, "count": N_BITSTRINGS, "index": BITSTRING_INDEX},
        "bits": [int(x) for x in bits], "open_tile": [int(q) for q in prob.open_tile],
        "n_paths": int(P), "partial_paths": PARTIAL,
        "full_re": [float(x) for x in total.real], "full_im": [float(x) for x in total.imag],
        "partial_re": [float(x) for x in partial.real], "partial_im": [float(x) for x in partial.imag],
        "seconds": round(time.time() - t0, 1), "cores": len(os.sched_getaffinity(0)),
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
