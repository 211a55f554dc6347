"""Figures of merit of §4.2 (Tables 5 and 6), in FP64.

TEST INFRASTRUCTURE (CPU oracle; never imported by the product path).

All measures compare an approximation C_hat (not the integer T) against the
orthonormal DCT C, with the first-order Markov covariance
R_x[i, j] = rho^|i-j|, rho = 0.95 (§4.2).

* total error energy     eps(C_hat) = pi * ||C - C_hat||_F^2
* mean square error      MSE(C_hat) = tr((C - C_hat) R_x (C - C_hat)^T) / 8
* coding gain            C_g, from the diagonal of R_y = C_hat R_x C_hat^T
* unified coding gain    C_g*, with rows of C_hat and of C_hat^{-1}
* transform efficiency   eta = sum |r_ii| / sum |r_ij| * 100
* circular statistics    mean angle, circular variance V, D_mod (Table 6)
"""
from __future__ import annotations

import numpy as np

from .matrices import dct_matrix

RHO = 0.95


def markov_covariance(n: int = 8, rho: float = RHO) -> np.ndarray:
    i = np.arange(n)
    return rho ** np.abs(i[:, None] - i[None, :]).astype(np.float64)


def total_error_energy(Chat: np.ndarray) -> float:
    C = dct_matrix(Chat.shape[0])
    return float(np.pi * np.sum((C - Chat) ** 2))


def matrix_mse(Chat: np.ndarray, rho: float = RHO) -> float:
    C = dct_matrix(Chat.shape[0])
    E = C - Chat
    Rx = markov_covariance(Chat.shape[0], rho)
    return float(np.trace(E @ Rx @ E.T) / Chat.shape[0])


def coding_gain(Chat: np.ndarray, rho: float = RHO) -> float:
    """C_g = 10 log10( mean(r_ii) / (prod r_ii ||c_i||^2)^(1/N) )."""
    N = Chat.shape[0]
    Rx = markov_covariance(N, rho)
    Ry = Chat @ Rx @ Chat.T
    r = np.diag(Ry)
    norms2 = np.sum(Chat**2, axis=1)
    return float(10.0 * np.log10(np.mean(r) / np.prod(r * norms2) ** (1.0 / N)))


def unified_coding_gain(Chat: np.ndarray, rho: float = RHO) -> float:
    """C_g* = 10 log10( prod_i 1 / (A_i B_i)^(1/N) ).

    A_i = su[(c_i c_i^T) o R_x] with c_i the i-th row of C_hat (as a column),
    B_i = ||g_i||^2 with g_i^T the i-th row of C_hat^{-1}, exactly as §4.2
    states.  For an orthogonal C_hat every B_i is 1 and C_g* equals C_g.
    """
    N = Chat.shape[0]
    Rx = markov_covariance(N, rho)
    G = np.linalg.inv(Chat)
    total = 0.0
    for i in range(N):
        c = Chat[i, :]
        A = float(np.sum(np.outer(c, c) * Rx))
        B = float(np.sum(G[i, :] ** 2))
        total += -np.log10(A * B) / N
    return float(10.0 * total)


def transform_efficiency(Chat: np.ndarray, rho: float = RHO) -> float:
    N = Chat.shape[0]
    Rx = markov_covariance(N, rho)
    Ry = Chat @ Rx @ Chat.T
    return float(np.sum(np.abs(np.diag(Ry))) / np.sum(np.abs(Ry)) * 100.0)


# --- circular statistics (§4.2, Table 6) ----------------------------------


def row_angles_to_e1(M: np.ndarray) -> np.ndarray:
    """theta_k = angle(a_k / ||a_k||, q), q = e_1 = [1,0,...,0]."""
    M = np.asarray(M, dtype=np.float64)
    a = M / np.linalg.norm(M, axis=1, keepdims=True)
    return np.arccos(np.clip(a[:, 0], -1.0, 1.0))


def circular_mean(theta: np.ndarray) -> float:
    """Mean direction by the case formula of §4.2 (radians, in [0, 2 pi))."""
    C = float(np.sum(np.cos(theta)))
    S = float(np.sum(np.sin(theta)))
    if C > 0 and S >= 0:
        return float(np.arctan(S / C))
    if C == 0 and S > 0:
        return float(np.pi / 2)
    if C < 0:
        return float(np.arctan(S / C) + np.pi)
    if C >= 0 and S < 0:
        if C == 0:
            return float(3 * np.pi / 2)
        return float(np.arctan(S / C) + 2 * np.pi)
    return float("nan")  # C = 0 and S = 0: undefined


def circular_variance(theta: np.ndarray) -> float:
    C = float(np.sum(np.cos(theta)))
    S = float(np.sum(np.sin(theta)))
    return 1.0 - np.sqrt(C * C + S * S) / len(theta)


def mean_circular_difference_mod(theta_c: np.ndarray, theta_t: np.ndarray) -> float:
    """D_mod = 1/N sum_i (pi - |pi - |theta_ci - theta_ti||)."""
    d = np.abs(theta_c - theta_t)
    return float(np.mean(np.pi - np.abs(np.pi - d)))


def mean_circular_difference(theta_c: np.ndarray, theta_t: np.ndarray) -> float:
    """D = 1/N^2 sum_i sum_j (pi - |pi - |theta_ci - theta_tj||)."""
    d = np.abs(theta_c[:, None] - theta_t[None, :])
    return float(np.mean(np.pi - np.abs(np.pi - d)))


def table5_row(Chat: np.ndarray) -> dict:
    return {
        "eps": total_error_energy(Chat),
        "mse": matrix_mse(Chat),
        "cg": coding_gain(Chat),
        "cg_star": unified_coding_gain(Chat),
        "eta": transform_efficiency(Chat),
    }


def table6_row(T: np.ndarray) -> dict:
    """Circular stats of the rows of T (degrees for the mean, radians for D_mod)."""
    th_t = row_angles_to_e1(T)
    th_c = row_angles_to_e1(dct_matrix(np.asarray(T).shape[0]))
    return {
        "mean_deg": float(np.degrees(circular_mean(th_t))),
        "var": circular_variance(th_t),
        "dmod": mean_circular_difference_mod(th_c, th_t),
    }
