"""The FP32 screen of the GPU angle search (§3, Eq. (6)) loses no candidate.

The kernels score candidates with FP32 cosines built from per-digit-group
tables (groups of 4 base-|P| digits, 3 when |P| >= 8): each group's partial
dot product with the exact DCT row is formed in FP64 and rounded to FP32,
the upper groups are summed first and group 0 last, and the sum is scaled by
the FP32 rounding of 1 / sqrt(||d||^2).  Only candidates within 1e-5 of the
FP32 maximum are re-scored in FP64.  That is exact if the FP32 cosine is
always within 5e-6 of the true one; the design bound is 9 * 2^-24 < 5.4e-7.
This test emulates that arithmetic in numpy float32 (round to nearest, the
same order of operations) over every candidate of several (N, P) and checks
the bound, with rows of the orthonormal N-point DCT-II as targets.
"""
import numpy as np
import pytest

SCREEN = 1e-5
BOUND = 9 * 2.0 ** -24


def dct_row(N, k):
    c = np.sqrt(1.0 / N) if k == 0 else np.sqrt(2.0 / N)
    return c * np.cos(np.pi * (2 * np.arange(N) + 1) * k / (2 * N))


def screen_errors(N, alphabet, k):
    vals = np.array(sorted(alphabet), dtype=np.int64)
    npv = len(vals)
    G = 4 if npv <= 7 else 3
    total = npv ** N
    idx = np.arange(total, dtype=np.int64)
    # digits, least significant first: digit t is coordinate N - 1 - t
    digits = np.empty((N, total), dtype=np.int64)
    rem = idx.copy()
    for t in range(N):
        digits[t] = rem % npv
        rem //= npv
    v = vals[digits]                       # v[t] = coordinate N - 1 - t
    crow_rev = dct_row(N, k)[::-1]         # coordinate order reversed like the digits
    groups = (N + G - 1) // G
    part64 = [np.zeros(total) for _ in range(groups)]
    for t in range(N):
        # the kernels fuse this multiply-add in FP64; the difference is ~1e-16
        part64[t // G] = part64[t // G] + crow_rev[t] * v[t]
    part32 = [p.astype(np.float32) for p in part64]
    up = np.zeros(total, dtype=np.float32)
    for g in range(1, groups):
        up = (up + part32[g]).astype(np.float32)
    d32 = (up + part32[0]).astype(np.float32)
    n2 = (v * v).sum(axis=0)
    ok = n2 > 0
    inv32 = (1.0 / np.sqrt(n2[ok].astype(np.float64))).astype(np.float32)
    cos32 = (d32[ok] * inv32).astype(np.float32).astype(np.float64)
    exact = (crow_rev[:, None] * v[:, ok]).sum(axis=0) / np.sqrt(n2[ok].astype(np.float64))
    return np.abs(cos32 - exact)


@pytest.mark.parametrize("N,alphabet", [(12, (-1, 0, 1)), (8, (-2, -1, 0, 1, 2)),
                                        (6, (-8, -4, -2, -1, 0, 1, 2, 4, 8)),
                                        (7, (-16, -3, 0, 1, 5, 9, 16))])
def test_fp32_cosine_error_is_within_the_screen(N, alphabet):
    for k in range(N):
        err = screen_errors(N, alphabet, k)
        assert err.max() <= BOUND, (N, alphabet, k, err.max())
    # the screen keeps every candidate within the tie tolerance of the maximum
    assert 2 * BOUND + 1e-12 < SCREEN
