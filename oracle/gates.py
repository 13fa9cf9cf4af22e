"""Exact gate matrices of the supremacy gate set (Sec. 2).  Oracle only.

Matrices act on the column vector (alpha_0, alpha_1) of one qubit; row-major.
"""
import numpy as np

_s2 = np.sqrt(0.5)  # correctly rounded 1/sqrt(2)

# Sec. 2: bit flip X, Hadamard H, T, X^{1/2}, Y^{1/2} as printed.
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
H = _s2 * np.array([[1, 1], [1, -1]], dtype=np.complex128)
# e^{i pi/4} = (1 + i)/sqrt(2), written with the correctly rounded 1/sqrt(2)
T = np.array([[1, 0], [0, _s2 + 1j * _s2]], dtype=np.complex128)
SQRT_X = 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128)
SQRT_Y = 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]], dtype=np.complex128)
# Sec. 2: CZ adds a -1 phase to |11>; symmetric in its two qubits.
CZ = np.diag(np.array([1, 1, 1, -1], dtype=np.complex128))

ONE_QUBIT = {"h": H, "t": T, "x_1_2": SQRT_X, "y_1_2": SQRT_Y, "x": X}
DIAGONAL = {"t", "cz"}
# Adjoints, for the inverse circuit (U^dagger undoes U).
INVERSE_NAME = {"h": "h", "t": "tdg", "x_1_2": "x_1_2dg", "y_1_2": "y_1_2dg",
                "cz": "cz", "x": "x", "tdg": "t", "x_1_2dg": "x_1_2", "y_1_2dg": "y_1_2"}
ONE_QUBIT.update({"tdg": T.conj().T, "x_1_2dg": SQRT_X.conj().T,
                  "y_1_2dg": SQRT_Y.conj().T})
DIAGONAL.add("tdg")


def matrix(name):
    """2x2 (or 4x4 for cz) complex128 matrix of a named gate."""
    if name == "cz":
        return CZ.copy()
    return ONE_QUBIT[name].copy()


def interleaved(m):
    """Row-major complex matrix as a flat float64 array (re, im, re, im, ...)."""
    m = np.ascontiguousarray(m, dtype=np.complex128)
    return m.reshape(-1).view(np.float64).copy()
