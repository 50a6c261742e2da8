"""Seeded synthetic inputs (circuits, bitstrings, problem descriptions).

Shared by the oracle, the tests and the bench; it holds no simulation
arithmetic of its own.
"""
from .circuits import (KINDS, KIND_ID, TWO_QUBIT, Circuit, Gate, Lattice, cz_counts,
                       diamond_lattice, grid_lattice, layer_edges,
                       random_bitstrings, random_circuit, two_qubit_counts)
from .problems import (Problem, c1_problem, c2_problem, c4_problem, diamond_problem,
                       grid_problem, grid_region_cuts, grid_region_ordering,
                       rotation_batch, row_major_ordering, workload_bitstrings)
