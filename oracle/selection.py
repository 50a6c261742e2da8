"""Fraction-f slice choice, sampling and norm estimates (oracle; test infrastructure only).

Methods, "Summing a fraction of the paths": summing a randomly chosen fraction
f of the paths yields a state of norm ~f and fidelity ~f (Eq. fidelity_1);
a single path p has fidelity <psi_p|psi_p> (Eq. fidelity_2).  The paper does
not say how the paths are drawn; the reading used here:
  n_f = max(1, floor(f * P + 1/2)) (ties round half up), capped at P;
  the chosen set is the first n_f entries of a Fisher-Yates shuffle of
  0..P-1 driven by SplitMix64(seed), j = next() mod (i + 1) for i = P-1..1;
  returned in ascending order.  No rescaling of the partial sums.
SplitMix64 follows its published definition (Steele, Lea, Flood 2014):
  x += 0x9E3779B97F4A7C15; z = x;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EB;  return z ^ (z >> 31).
"""
from __future__ import annotations

import math
from typing import List

import numpy as np

_M64 = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.x = seed & _M64

    def next(self) -> int:
        self.x = (self.x + 0x9E3779B97F4A7C15) & _M64
        z = self.x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)


def n_selected(fidelity: float, P: int) -> int:
    return int(min(P, max(1, math.floor(fidelity * P + 0.5))))


def select_slices(P: int, fidelity: float, seed: int) -> List[int]:
    a = list(range(P))
    rng = SplitMix64(seed)
    for i in range(P - 1, 0, -1):
        j = rng.next() % (i + 1)
        a[i], a[j] = a[j], a[i]
    return sorted(a[:n_selected(fidelity, P)])


def frugal_sample(amps: np.ndarray, n_qubits: int, M: float, seed: int) -> np.ndarray:
    """Frugal rejection sampling over batches (Methods, "Fast sampling technique").

    For each batch (row) the entries are visited in a uniformly random order
    and the first one with u < p N / M is accepted (p = |amp|^2, N = 2^n); at
    most one sample per batch, -1 if the batch is exhausted.  Randomness, as
    specified for both implementations: a SplitMix64 stream per batch from
    seed + b * 0xD1B54A32D192ED03; visiting order by a forward Fisher-Yates
    walk (step k swaps entries k and k + x mod (n_c - k)); u = (x >> 11) 2^-53.
    """
    amps = np.atleast_2d(np.asarray(amps, dtype=np.complex128))
    n_b, n_c = amps.shape
    scale = float(2.0 ** n_qubits) / M
    out = np.full(n_b, -1, dtype=np.int32)
    for b in range(n_b):
        rng = SplitMix64((seed + b * 0xD1B54A32D192ED03) & _M64)
        order = list(range(n_c))
        for k in range(n_c):
            j = k + rng.next() % (n_c - k)
            order[k], order[j] = order[j], order[k]
            idx = order[k]
            a = amps[b, idx]
            p = a.real * a.real + a.imag * a.imag
            u = (rng.next() >> 11) * 2.0 ** -53
            if u < p * scale:
                out[b] = idx
                break
    return out


def overlap_fidelity(psi_exact: np.ndarray, psi_partial: np.ndarray) -> float:
    """|<psi|psi~>|^2 / <psi~|psi~> (Eq. fidelity_1 / fidelity_2)."""
    a = np.asarray(psi_exact).reshape(-1)
    b = np.asarray(psi_partial).reshape(-1)
    return float(abs(np.vdot(a, b)) ** 2 / np.vdot(b, b).real)


STREAM_STEP = 0xD1B54A32D192ED03


def fidelity_samples(batch_bits: np.ndarray, accepted: np.ndarray, tile, fidelity: float,
                     seed: int, n_samples: int):
    """Fidelity-f samples from perfect-fidelity amplitudes (Methods, "Fraction
    of perfect fidelity amplitudes"): a fidelity-f circuit outputs
    rho = f |psi><psi| + (1 - f) I / N, so each sample is, with probability f,
    an exact sample of |psi> and otherwise a uniformly random bitstring.

    Exact samples are the batches that frugal rejection sampling accepted
    (accepted[b] = tile index j, or -1), used in batch order; the k-th exact
    sample takes the k-th accepted batch: its bits batch_bits[b] with tile
    qubit t set to bit (|tile| - 1 - t) of j.  Randomness, as specified for
    both implementations: sample i runs its own SplitMix64 stream from
    seed + i * 0xD1B54A32D192ED03; the first draw x gives u = (x >> 11) 2^-53
    and the sample is exact when u < f; a uniform sample takes qubit q from
    bit 63 - (q mod 64) of draw number 1 + q div 64.

    Returns (samples uint8 [n_samples, n], source int32 [n_samples] with the
    batch index of an exact sample, -1 for a uniform one and -2 for an exact
    one beyond the accepted batches (its bits are zero), n_exact).
    """
    batch_bits = np.asarray(batch_bits, dtype=np.uint8)
    accepted = np.asarray(accepted, dtype=np.int64).reshape(-1)
    n = batch_bits.shape[1] if batch_bits.ndim == 2 else int(len(batch_bits))
    nt = len(tile)
    pool = [b for b in range(len(accepted)) if accepted[b] >= 0]
    samples = np.zeros((n_samples, n), dtype=np.uint8)
    source = np.full(n_samples, -1, dtype=np.int32)
    k = 0
    for i in range(n_samples):
        rng = SplitMix64((seed + i * STREAM_STEP) & _M64)
        u = (rng.next() >> 11) * 2.0 ** -53
        if u < fidelity:
            if k < len(pool):
                b = pool[k]
                source[i] = b
                samples[i] = batch_bits[b]
                j = int(accepted[b])
                for t, q in enumerate(tile):
                    samples[i, q] = (j >> (nt - 1 - t)) & 1
            else:
                source[i] = -2
            k += 1
        else:
            w = 0
            for q in range(n):
                if q % 64 == 0:
                    w = rng.next()
                samples[i, q] = (w >> (63 - q % 64)) & 1
    return samples, source, k


def linear_xeb(probabilities: np.ndarray, n_qubits: int) -> float:
    """Linear cross-entropy fidelity estimate N <p(x)> - 1 over sampled x."""
    return float((2.0 ** n_qubits) * np.mean(np.asarray(probabilities)) - 1.0)
