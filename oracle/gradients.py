"""Angle gradients of amplitudes (oracle; test infrastructure only).

The paper has no gradients; they follow from the gate definitions.  With
R_P(t) = cos(t/2) I - i sin(t/2) P, dR_P/dt = (1/2) R_P(t + pi), and since each
angle enters exactly one gate, the amplitude is linear in that gate, so
  d amp / d t_g = (1/2) amp(t with t_g -> t_g + pi)      (exact shift rule).
For complex outputs a and a real upstream cotangent g (complex), the gradient
of the real loss L = Re sum_j conj(g_j) a_j is sum_j Re(conj(g_j) d a_j/d t).

Three independent routes are provided: the shift rule (any amplitude
routine), central finite differences, and a state-vector adjoint
(forward state, backward co-state) for small circuits.
"""
from __future__ import annotations

from typing import Callable, Optional, Sequence

import numpy as np

from . import gates as G
from .statevector import _apply_1q, _apply_2q, _cz


def shift_rule(amp_fn: Callable[[np.ndarray], np.ndarray], angles: np.ndarray,
               params: Sequence[int]) -> np.ndarray:
    """[len(params), ...] d amp / d angle via the exact shift rule."""
    out = []
    for p in params:
        th = np.array(angles, dtype=np.float64, copy=True)
        th[p] += np.pi
        out.append(0.5 * amp_fn(th))
    return np.stack(out)


def finite_difference(amp_fn, angles: np.ndarray, params: Sequence[int],
                      h: float = 1e-5) -> np.ndarray:
    out = []
    for p in params:
        tp = np.array(angles, dtype=np.float64, copy=True)
        tm = tp.copy()
        tp[p] += h
        tm[p] -= h
        out.append((amp_fn(tp) - amp_fn(tm)) / (2.0 * h))
    return np.stack(out)


def loss_gradient(damp: np.ndarray, upstream: np.ndarray) -> np.ndarray:
    """sum over amplitude entries of Re(conj(g) * d amp / d t) per parameter."""
    d = damp.reshape(damp.shape[0], -1)
    g = np.asarray(upstream).reshape(-1)
    return np.real(np.conj(g)[None, :] * d).sum(axis=1)


def statevector_adjoint(circ, bitstrings: np.ndarray, tile: Sequence[int],
                        upstream: np.ndarray, angles: Optional[np.ndarray] = None
                        ) -> np.ndarray:
    """Gradient of L = Re sum_j conj(g_j) amp_j w.r.t. every angle, adjoint method.

    phi_k = G_k ... G_1 |0>, chi = sum_j g_j |x_j> propagated backwards;
    d amp/d t_k contributes <chi_k| dG_k/dt |phi_{k-1}>.
    """
    n = circ.n
    angles = circ.angles if angles is None else np.asarray(angles, dtype=np.float64)
    seq = sorted(circ.gates, key=lambda g: g.cycle)
    psi = np.zeros((2,) * n, dtype=np.complex128)
    psi[(0,) * n] = 1.0
    for g in seq:
        if g.kind == "CZ":
            psi = _cz(psi, g.q0, g.q1)
        elif g.kind == "ISWAP":
            psi = _apply_2q(psi, G.ISWAP, min(g.q0, g.q1), max(g.q0, g.q1))
        else:
            psi = _apply_1q(psi, G.single_qubit_matrix(g.kind, angles, g.param), g.q0)
    chi = np.zeros_like(psi)
    bitstrings = np.atleast_2d(bitstrings)
    up = np.asarray(upstream).reshape(len(bitstrings), -1)
    nt = len(tile)
    for i, b in enumerate(bitstrings):
        x = [int(v) for v in b]
        for j in range(1 << nt):
            for t, q in enumerate(tile):
                x[q] = (j >> (nt - 1 - t)) & 1
            chi[tuple(x)] += up[i, j]
    grad = np.zeros(circ.n_params, dtype=np.float64)
    for g in reversed(seq):
        if g.kind == "CZ":
            psi = _cz(psi, g.q0, g.q1)          # CZ is its own inverse
            chi = _cz(chi, g.q0, g.q1)
            continue
        if g.kind == "ISWAP":                   # step back with U^dagger
            a, b = min(g.q0, g.q1), max(g.q0, g.q1)
            psi = _apply_2q(psi, G.ISWAP.conj().T, a, b)
            chi = _apply_2q(chi, G.ISWAP.conj().T, a, b)
            continue
        U = G.single_qubit_matrix(g.kind, angles, g.param)
        psi = _apply_1q(psi, U.conj().T, g.q0)  # phi_{k-1}
        if g.param >= 0:
            dU = 0.5 * G.rotation(g.kind, float(angles[g.param]) + np.pi)
            val = np.vdot(chi, _apply_1q(psi, dU, g.q0))   # <chi| dU phi> = sum conj(chi) ...
            # d amp_j = <x_j|...dU...|0>; L = Re sum conj(g_j) amp_j and
            # chi = sum g_j |x_j>, so dL = Re <chi| dU phi>.
            grad[g.param] += np.real(val)
        chi = _apply_1q(chi, U.conj().T, g.q0)
    return grad
