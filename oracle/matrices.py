"""Transform matrices of the paper, restated for the oracle (FP64 / exact ints).

TEST INFRASTRUCTURE: this package is the CPU oracle.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The product path never does.

Contents
--------
* ``dct_matrix()``      -- the exact 8-point DCT-II matrix C (§2).  The paper
  prints C with entries gamma_k = cos(2*pi*(k+1)/32) and no scale factor; that
  printed matrix has row norms 2, i.e. it is twice the orthonormal DCT.  Only
  the orthonormal C reproduces Table 5, so this returns C/2 written out from
  the cosine definition C[k, j] = c_k cos(pi (2j+1) k / 16).
* ``T1``, ``T2``        -- the two new low-complexity matrices found by the
  greedy search over D2 (§4.1).
* ``T_RDCT``, ``T_BAS2008B``, ``T_LO``, ``T6``, ``T4`` -- literature matrices
  of Table 2 (LO has entries +-1/2 and is kept as a float matrix).
* ``A1..A4``, ``D``     -- the sparse factors of T1 (§5.1, T1 = D A4 A3 A2 A1).
* ``approximation(T)``  -- C_hat = S T with S = sqrt((T T^T)^-1), Eq. (1)-(2).
"""
from __future__ import annotations

import numpy as np

# --- Exact DCT (§2) --------------------------------------------------------


def dct_matrix(n: int = 8) -> np.ndarray:
    """Orthonormal DCT-II, C[k, j] = c_k cos(pi (2j+1) k / (2n)).

    c_0 = sqrt(1/n), c_k = sqrt(2/n).  For n = 8 this is the matrix printed in
    §2 (gamma_k = cos(2 pi (k+1)/32)) divided by 2.
    """
    k = np.arange(n)[:, None].astype(np.float64)
    j = np.arange(n)[None, :].astype(np.float64)
    C = np.cos(np.pi * (2.0 * j + 1.0) * k / (2.0 * n))
    C[0, :] *= np.sqrt(1.0 / n)
    C[1:, :] *= np.sqrt(2.0 / n)
    return C


def printed_dct_matrix() -> np.ndarray:
    """The DCT matrix exactly as printed in §2 (gamma symbols, no 1/2 factor).

    Row k lists gamma indices with signs; gamma_g = cos(2 pi (g+1) / 32).
    Kept so that a test can show the printed matrix equals 2 * dct_matrix().
    """
    g = lambda i: np.cos(2.0 * np.pi * (i + 1) / 32.0)  # noqa: E731
    rows = [
        [(+1, 3)] * 8,
        [(+1, 0), (+1, 2), (+1, 4), (+1, 6), (-1, 6), (-1, 4), (-1, 2), (-1, 0)],
        [(+1, 1), (+1, 5), (-1, 5), (-1, 1), (-1, 1), (-1, 5), (+1, 5), (+1, 1)],
        [(+1, 2), (-1, 6), (-1, 0), (-1, 4), (+1, 4), (+1, 0), (+1, 6), (-1, 2)],
        [(+1, 3), (-1, 3), (-1, 3), (+1, 3), (+1, 3), (-1, 3), (-1, 3), (+1, 3)],
        [(+1, 4), (-1, 0), (+1, 6), (+1, 2), (-1, 2), (-1, 6), (+1, 0), (-1, 4)],
        [(+1, 5), (-1, 1), (+1, 1), (-1, 5), (-1, 5), (+1, 1), (-1, 1), (+1, 5)],
        [(+1, 6), (-1, 4), (+1, 2), (-1, 0), (+1, 0), (-1, 2), (+1, 4), (-1, 6)],
    ]
    return np.array([[s * g(i) for (s, i) in row] for row in rows], dtype=np.float64)


# --- Low-complexity matrices ----------------------------------------------

# §4.1: the two matrices obtained from the search over D2 = {0,+-1,+-2}^8.
T1 = np.array(
    [
        [1, 1, 1, 1, 1, 1, 1, 1],
        [2, 2, 1, 0, 0, -1, -2, -2],
        [2, 1, -1, -2, -2, -1, 1, 2],
        [1, 0, -2, -2, 2, 2, 0, -1],
        [1, -1, -1, 1, 1, -1, -1, 1],
        [2, -2, 0, 1, -1, 0, 2, -2],
        [1, -2, 2, -1, -1, 2, -2, 1],
        [0, -1, 2, -2, 2, -2, 1, 0],
    ],
    dtype=np.int64,
)

T2 = np.array(
    [
        [1, 1, 1, 1, 1, 1, 1, 1],
        [2, 1, 2, 0, 0, -2, -1, -2],
        [2, 1, -1, -2, -2, -1, 1, 2],
        [2, 0, -2, -1, 1, 2, 0, -2],
        [1, -1, -1, 1, 1, -1, -1, 1],
        [1, -2, 0, 2, -2, 0, 2, -1],
        [1, -2, 2, -1, -1, 2, -2, 1],
        [0, -2, 1, -2, 2, -1, 2, 0],
    ],
    dtype=np.int64,
)

# Table 2 (literature matrices).
T_RDCT = np.array(
    [
        [1, 1, 1, 1, 1, 1, 1, 1],
        [1, 1, 1, 0, 0, -1, -1, -1],
        [1, 0, 0, -1, -1, 0, 0, 1],
        [1, 0, -1, -1, 1, 1, 0, -1],
        [1, -1, -1, 1, 1, -1, -1, 1],
        [1, -1, 0, 1, -1, 0, 1, -1],
        [0, -1, 1, 0, 0, 1, -1, 0],
        [0, -1, 1, -1, 1, -1, 1, 0],
    ],
    dtype=np.int64,
)

T_BAS2008B = np.array(
    [
        [1, 1, 1, 1, 1, 1, 1, 1],
        [1, 1, 1, 0, 0, -1, -1, -1],
        [1, 1, -1, -1, -1, -1, 1, 1],
        [1, 0, -1, 0, 0, 1, 0, -1],
        [1, -1, -1, 1, 1, -1, -1, 1],
        [1, -1, 1, 0, 0, -1, 1, -1],
        [1, -1, 1, -1, -1, 1, -1, 1],
        [1, -1, 1, -1, 1, -1, 1, -1],
    ],
    dtype=np.int64,
)

_h = 0.5
T_LO = np.array(
    [
        [1, 1, 1, 1, 1, 1, 1, 1],
        [1, 1, 1, 0, 0, -1, -1, -1],
        [1, _h, -_h, -1, -1, -_h, _h, 1],
        [1, 0, -1, -1, 1, 1, 0, -1],
        [1, -1, -1, 1, 1, -1, -1, 1],
        [1, -1, 0, 1, -1, 0, 1, -1],
        [_h, -1, 1, -_h, -_h, 1, -1, _h],
        [0, -1, 1, -1, 1, -1, 1, 0],
    ],
    dtype=np.float64,
)

T6 = np.array(
    [
        [1, 1, 1, 1, 1, 1, 1, 1],
        [2, 1, 1, 0, 0, -1, -1, -2],
        [2, 1, -1, -2, -2, -1, 1, 2],
        [1, 0, -2, -1, 1, 2, 0, -1],
        [1, -1, -1, 1, 1, -1, -1, 1],
        [1, -2, 0, 1, -1, 0, 2, -1],
        [1, -2, 2, -1, -1, 2, -2, 1],
        [0, -1, 1, -2, 2, -1, 1, 0],
    ],
    dtype=np.int64,
)

T4 = np.array(
    [
        [1, 1, 1, 1, 1, 1, 1, 1],
        [1, 1, 1, 0, 0, -1, -1, -1],
        [1, 1, -1, -1, -1, -1, 1, 1],
        [1, 0, -1, -1, 1, 1, 0, -1],
        [1, -1, -1, 1, 1, -1, -1, 1],
        [1, -1, 0, 1, -1, 0, 1, -1],
        [1, -1, 1, -1, -1, 1, -1, 1],
        [0, -1, 1, -1, 1, -1, 1, 0],
    ],
    dtype=np.int64,
)

# --- Sparse factorisation of T1 (§5.1) -----------------------------------

A1 = np.array(
    [
        [1, 0, 0, 0, 0, 0, 0, 1],
        [0, 1, 0, 0, 0, 0, 1, 0],
        [0, 0, 1, 0, 0, 1, 0, 0],
        [0, 0, 0, 1, 1, 0, 0, 0],
        [0, 0, 0, 1, -1, 0, 0, 0],
        [0, 0, 1, 0, 0, -1, 0, 0],
        [0, 1, 0, 0, 0, 0, -1, 0],
        [1, 0, 0, 0, 0, 0, 0, -1],
    ],
    dtype=np.float64,
)
A2 = np.array(
    [
        [1, 0, 0, 1, 0, 0, 0, 0],
        [0, 1, 1, 0, 0, 0, 0, 0],
        [0, 1, -1, 0, 0, 0, 0, 0],
        [1, 0, 0, -1, 0, 0, 0, 0],
        [0, 0, 0, 0, 1, 0, 0, 0],
        [0, 0, 0, 0, 0, 1, 0, 0],
        [0, 0, 0, 0, 0, 0, 1, 0],
        [0, 0, 0, 0, 0, 0, 0, 1],
    ],
    dtype=np.float64,
)
A3 = np.eye(8)
A3[0, :2] = [1, 1]
A3[1, :2] = [1, -1]
A4 = np.array(
    [
        [1, 0, 0, 0, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, _h, 1, 1],
        [0, 0, 1, 2, 0, 0, 0, 0],
        [0, 0, 0, 0, -1, -1, 0, _h],
        [0, 1, 0, 0, 0, 0, 0, 0],
        [0, 0, 0, 0, _h, 0, -1, 1],
        [0, 0, -2, 1, 0, 0, 0, 0],
        [0, 0, 0, 0, -1, 1, -_h, 0],
    ],
    dtype=np.float64,
)
D = np.diag([1.0, 2.0, 1.0, 2.0, 1.0, 2.0, 1.0, 2.0])


# --- Approximation model, Eq. (1)-(2) -------------------------------------


def sqrtm_spd(M: np.ndarray) -> np.ndarray:
    """Principal square root of a symmetric positive definite matrix."""
    w, V = np.linalg.eigh(M)
    return (V * np.sqrt(w)) @ V.T


def scaling_matrix(T: np.ndarray) -> np.ndarray:
    """S = sqrt((T T^T)^-1), Eq. (2)."""
    T = np.asarray(T, dtype=np.float64)
    return sqrtm_spd(np.linalg.inv(T @ T.T))


def approximation(T: np.ndarray) -> np.ndarray:
    """C_hat = S . T, Eq. (1)."""
    T = np.asarray(T, dtype=np.float64)
    return scaling_matrix(T) @ T


def row_norms_sq(T: np.ndarray) -> np.ndarray:
    """n_k = diag(T T^T); for an orthogonal T, S = diag(1/sqrt(n_k))."""
    T = np.asarray(T)
    return np.einsum("ij,ij->i", T, T)


NAMED = {
    "T1": T1,
    "T2": T2,
    "RDCT": T_RDCT,
    "BAS2008B": T_BAS2008B,
    "LO": T_LO,
    "T6": T6,
    "T4": T4,
}
