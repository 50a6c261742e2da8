"""Gate matrices in complex128 (oracle; test infrastructure only).

The paper names the gates (Methods, "Revised set of RQCs": H, T, X^1/2,
Y^1/2 and CZ) without writing their matrices.  The reading used here:
  H      = (1/sqrt 2) [[1, 1], [1, -1]]
  T      = diag(1, e^{i pi/4})
  X^1/2  = principal square root of X = 1/2 [[1+i, 1-i], [1-i, 1+i]]
  Y^1/2  = principal square root of Y = 1/2 [[1+i, -1-i], [1+i, 1+i]]
  CZ     = diag(1, 1, 1, -1)
  R_P(t) = exp(-i t P / 2) = cos(t/2) I - i sin(t/2) P   for P in {X, Y, Z}
iSWAP is written out in the paper (Methods, "Revised set of RQCs") as
|00><00| + |11><11| + i|01><10| + i|10><01|, first qubit = lower index.
Pinned in tests by: X^1/2 squared = X, Y^1/2 squared = Y, T^2 = diag(1, i),
H^2 = I, unitarity, R_X(pi) = -iX, R_P(t) against scipy's expm, and the
iSWAP split summing back to the ket-bra definition with operator-Schmidt
rank 4 (Methods, "Overview of the simulator").
"""
import numpy as np

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)
T = np.diag([1.0, np.exp(1j * np.pi / 4)]).astype(np.complex128)
SX = 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128)
SY = 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]], dtype=np.complex128)
CZ = np.diag([1.0, 1.0, 1.0, -1.0]).astype(np.complex128)

ISWAP = np.array([[1, 0, 0, 0],
                  [0, 0, 1j, 0],
                  [0, 1j, 0, 0],
                  [0, 0, 0, 1]], dtype=np.complex128)

PAULI = {"RX": X, "RY": Y, "RZ": Z}


def rotation(kind: str, theta: float) -> np.ndarray:
    """R_P(theta) = cos(theta/2) I - i sin(theta/2) P."""
    return np.cos(theta / 2.0) * I2 - 1j * np.sin(theta / 2.0) * PAULI[kind]


def single_qubit_matrix(kind: str, angles: np.ndarray, param: int) -> np.ndarray:
    if kind == "H":
        return H
    if kind == "T":
        return T
    if kind == "SX":
        return SX
    if kind == "SY":
        return SY
    if kind in PAULI:
        return rotation(kind, float(angles[param]))
    raise ValueError(f"not a single-qubit gate: {kind}")


def cz_half(role: str, k: int) -> np.ndarray:
    """One half of the CZ Schmidt decomposition (-1)^{ab} = sum_k d_{a,k} (-1)^{k b}.

    The paper gives the Schmidt rank (2, Methods "Overview of the simulator")
    but not the split; reading: the lower-index qubit carries the projector
    |k><k| ("proj"), the higher-index qubit carries Z^k ("z").
    """
    if role == "proj":
        return np.diag([1.0 if k == 0 else 0.0, 1.0 if k == 1 else 0.0]).astype(np.complex128)
    return np.diag([1.0, (-1.0) ** k]).astype(np.complex128)


def iswap_half(role: str, k: int) -> np.ndarray:
    """One term of the iSWAP operator-Schmidt split iSWAP = sum_k A_k (x) B_k.

    The paper gives the rank (4, Methods "Overview of the simulator") but not
    the split.  Reading: in the Pauli basis iSWAP = (I I + Z Z)/2 +
    i (X X + Y Y)/2, so with P_k = (I, Z, X, Y)[k] the lower-index qubit
    ("a") carries A_k = P_k and the higher-index qubit ("b") carries
    B_k = c_k P_k, c = (1/2, 1/2, i/2, i/2).  k is a 2-bit bond value, its
    high bit first in the bond multi-index.
    """
    P = (I2, Z, X, Y)[k]
    if role == "a":
        return P.copy()
    return (0.5, 0.5, 0.5j, 0.5j)[k] * P
