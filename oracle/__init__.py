"""FP64 CPU oracle for the RQC amplitude path -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the bench's CPU-baseline leg may import
this package.  The product path (the CUDA library and its Python binding)
never imports, links or executes anything here, and this package imports
nothing from the product; the two share only the seeded input generators in
``qflex_inputs`` (which hold no simulation arithmetic).

Contents (each function cites the passage of the paper it follows):
  gates        -- gate matrices (Methods, "Revised set of RQCs")
  statevector  -- brute-force state-vector amplitudes (the plain definition
                  amp(x) = <x|U|0^n>), including cut-slice variants
  network      -- grid tensors and labelled pairwise contraction with cuts,
                  open tile and partial slice sums (Methods, "Overview of the
                  simulator", "Contraction of the 3D tensor network",
                  "Cutting indexes", "Fast sampling technique")
  permute      -- index permutation (row-major) and the paper's left/right
                  move decomposition ("Cache-efficient index permutations")
  gradients    -- angle gradients by the exact shift rule, central finite
                  differences and a state-vector adjoint
  selection    -- SplitMix64 / Fisher-Yates choice of the fraction-f slices
                  ("Summing a fraction of the paths") and norm estimates

Parity status: every function is pinned by a `-m "not gpu"` test against a
closed form, a brute-force route or a worked example of the paper, except the
exact Google CZ layer order and the Bristlecone device coordinates (figure
only in the paper; "parity unpinned" -- immaterial to parity because both
sides consume the same generated circuit).
"""
