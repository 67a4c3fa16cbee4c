"""Test-side D3Q19 table, typed independently from the paper (Sec. 2.1).

Used only to build inputs (equilibrium fields) and to read results; it is
neither the oracle's table nor the kernels'.
"""
import numpy as np

C = np.array([
    (0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
    (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
    (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)], dtype=np.float64)
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
OPP = np.array([0] + [q + 1 if q % 2 == 1 else q - 1 for q in range(1, 19)])


def equilibrium(rho, U):
    """Eq. 5 for one cell: rho scalar, U length-3."""
    U = np.asarray(U, dtype=np.float64)
    cu = C @ U
    return W * (rho + 3.0 * cu + 4.5 * cu * cu - 1.5 * (U @ U))


def uniform_field(fq, shape):
    """Field f[q][z][y][x] holding the 19 values fq in every cell."""
    return np.broadcast_to(np.asarray(fq)[:, None, None, None], (19,) + tuple(shape)).copy()
