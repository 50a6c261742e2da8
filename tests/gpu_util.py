"""Helpers shared by the GPU tests (error metrics; no simulation arithmetic)."""
import numpy as np

# Tolerances on the amplitude error metric below.
# fp32 (24-bit products) is gated at 1e-5; the 3-term split forms (tf32x3 and
# scaled fp16x3: ~22 bits, bf16x3: ~16 bits) at 1e-4.
TOL = {"fp32": 1e-5, "tf32x3": 1e-4, "bf16x3": 1e-4, "fp16x3": 1e-4}


def amp_error(got, ref, n_qubits, f_eff=1.0):
    """max_j |a_j - r_j| / max(|r_j|, sqrt(f_eff 2^-n)).

    The floor is the typical Porter-Thomas amplitude magnitude of a
    fidelity-f_eff state, so near-zero amplitudes do not dominate.
    """
    got = np.asarray(got).reshape(-1)
    ref = np.asarray(ref).reshape(-1)
    floor = np.sqrt(f_eff * 2.0 ** (-n_qubits))
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor)))


def gemm_error(got, ref):
    """max |C - R| / max |R| for a GEMM on random inputs."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
