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


def jam(T_half: np.ndarray, lower_add: str = "I,-Ibar") -> np.ndarray:
    """The JAM step of §6.2, Eq. (jam), without its 1/sqrt(2) (merged into the
    scaling): T_(N) = M_per [T_(N/2) 0; 0 T_(N/2)] M_add.

    M_per is built from P_{N-1, N/2}, whose even rows i are row i/2 of the
    identity and odd rows zero; its printed block layout places the
    (N-1) x (N/2) block P beside a 1 x (N/2) zero block, read here as block
    columns [P; 0] and [0; P]: the N x N permutation taking row 2i from the
    first copy of T_(N/2) and row 2i + 1 from the second.

    M_add's upper block row is [I, Ibar] (Ibar the counter-identity).  Its
    printed lower block row [Ibar, -I] does not give the matrices the paper
    prints after the recursion; [I, -Ibar] does (the two differ only in the
    signs of the rows built from antisymmetric rows of T_(N/2), which leaves
    the codec's reconstruction unchanged).  ``lower_add`` selects "I,-Ibar"
    (default, the printed matrices) or "Ibar,-I" (the printed formula)."""
    T_half = np.asarray(T_half, dtype=np.int64)
    h = T_half.shape[0]
    N = 2 * h
    I = np.eye(h, dtype=np.int64)
    Ibar = I[::-1]
    lower = np.hstack([I, -Ibar]) if lower_add == "I,-Ibar" else np.hstack([Ibar, -I])
    M_add = np.vstack([np.hstack([I, Ibar]), lower])
    P = np.zeros((N - 1, h), dtype=np.int64)
    for i in range(0, N - 1, 2):
        P[i] = I[i // 2]
    z = np.zeros((1, h), dtype=np.int64)
    M_per = np.hstack([np.vstack([P, z]), np.vstack([z, P])])
    blk = np.block([[T_half, np.zeros((h, h), np.int64)], [np.zeros((h, h), np.int64), T_half]])
    return M_per @ blk @ M_add


def jam_cost(N: int) -> tuple[int, int]:
    """(additions, shifts) of the JAM transform from T1 (§6.2): twice the
    half-size transform's counts plus N additions for M_add; T1 itself has
    24 additions and 6 shifts (§5.1)."""
    if N == 8:
        return 24, 6
    a, s = jam_cost(N // 2)
    return 2 * a + N, 2 * s


T16 = jam(T1)
T32 = jam(T16)

NAMED = {
    "T1": T1,
    "T2": T2,
    "RDCT": T_RDCT,
    "BAS2008B": T_BAS2008B,
    "LO": T_LO,
    "T6": T6,
    "T4": T4,
}
