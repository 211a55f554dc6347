"""Integer identities the CUDA epilogues rely on, checked on the CPU.

The reconstruction of §6.1 (reading R5: round half away from zero, then
clamp) is evaluated on the GPU through the doubled inverse 2N and a division
by 2 L^2 done with a multiply-high by a constant.  These tests restate each
identity with its range of validity and check it on exhaustive or dense sets,
ties (N = +-L^2 / 2 mod L^2) included.
"""
import numpy as np

L2 = 360 * 360            # L^2 of T1 (L = lcm(8, 18, 20) = 360)
D = 2 * L2
MAGIC = 1085937411        # the 8x8 kernels' division constant


def half_away(N, L2=L2):
    return np.sign(N) * ((np.abs(N) + L2 // 2) // L2)


def mulhi_hi16(a, m):
    """Upper 16 bits of the signed 32 x 32 high product: floor(a m / 2^48)."""
    return ((a * m) >> 32) >> 16


def dense_N(lim, L2=L2, seed=0):
    rng = np.random.default_rng(seed)
    ties = np.arange(-300, 300, dtype=np.int64) * L2
    return np.concatenate([rng.integers(-lim, lim, 1_000_000), np.arange(-4 * L2, 4 * L2),
                           ties + L2 // 2, ties - L2 // 2, ties]).astype(np.int64)


def test_u8_epilogue_rounds_half_away_for_nonnegative_N():
    # u8: x' = floor((2N + L^2) / (2 L^2)) from the high half of mulhi; valid on
    # [0, 256 * 2 L^2) (above clamps to 255) and negative for negative dividends
    N = dense_N(256 * L2)
    a = 2 * N + L2
    q = mulhi_hi16(a, MAGIC)
    pos = N >= 0
    assert np.array_equal(np.clip(q[pos], 0, 255), np.clip(half_away(N[pos]), 0, 255))
    assert (q[a < 0] < 0).all()


def test_int16_epilogue_offset_form():
    # int16: floor((2N + L^2 - [N < 0] + 2048 * 2 L^2) / (2 L^2)) - 2048 equals
    # round-half-away for both signs; the dividend stays in [0, 1.27e9) for
    # |N| <= 255 * 8 * L^2 (orthogonal-projection bound), where MAGIC is exact
    lim = 255 * 8 * L2
    N = dense_N(lim)
    N = N[np.abs(N) <= lim]
    a = 2 * N - (N < 0) + L2 + 2048 * D
    assert a.min() >= 0 and a.max() < 1.27e9
    q = mulhi_hi16(a, MAGIC) - 2048
    assert np.array_equal(np.clip(q, -255, 255), np.clip(half_away(N), -255, 255))


def test_magic_is_exact_on_its_range():
    # floor(a / (2 L^2)) == (a * MAGIC) >> 48 for 0 <= a < 1.27e9 (sampled
    # densely, plus every multiple of 2 L^2 and its predecessor)
    a = np.concatenate([np.arange(0, 1_270_000_000, 997, dtype=np.int64),
                        np.arange(0, 1_270_000_000, D, dtype=np.int64),
                        np.arange(D - 1, 1_270_000_000, D, dtype=np.int64)])
    assert np.array_equal(mulhi_hi16(a, MAGIC), a // D)


def test_jam16_lane_constant_is_exact_on_the_clamp_window():
    # 16x16 JAM blocks (L = 720): m16 = ceil(2^48 / (2 L^2)) gives
    # floor(a / (2 L^2)) in the upper half of the signed high product for
    # 0 <= a <= 256 * 2 L^2, and a negative upper half below 0
    L2j = 720 * 720
    d = 2 * L2j
    m16 = ((1 << 48) + d - 1) // d
    assert m16 < 2 ** 31
    limit = 256 * d
    a = np.concatenate([np.arange(0, limit + 1, 101, dtype=np.int64),
                        np.arange(0, limit + 1, d, dtype=np.int64),
                        np.arange(d - 1, limit + 1, d, dtype=np.int64)])
    assert np.array_equal(mulhi_hi16(a, m16), a // d)
    neg = np.arange(-(2 ** 31) + 128 * d, 0, 100_003, dtype=np.int64)
    assert (mulhi_hi16(neg, m16) < 0).all()
