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
    # int16: q = floor((2N + L^2 - [N < 0] + 255 * 2 L^2) / (2 L^2)) by the
    # multiply-high, clamped to [0, 510] (min.relu.s16x2), minus 255 (vsub2),
    # equals round-half-away clamped to [-255, 255] for both signs.  For
    # |N| <= 255 * 8 * L^2 (orthogonal-projection bound) the dividend lies in
    # [-3569 L^2, 4591 L^2]: below 1.27e9 where MAGIC is exact, and a negative
    # dividend gives a negative q (clamped to 0).  The upper halves fit int16.
    lim = 255 * 8 * L2
    N = dense_N(lim)
    N = N[np.abs(N) <= lim]
    a = 2 * N - (N < 0) + L2 + 255 * D
    assert a.max() < 1.27e9
    q = mulhi_hi16(a, MAGIC)
    assert np.abs(q).max() < 2 ** 15
    assert (q[a < 0] < 0).all()
    x = np.clip(q, 0, 510) - 255
    assert np.array_equal(x, np.clip(half_away(N), -255, 255))


def test_int16_packed_sse_terms():
    # vabsdiffs2 of an int16 sample pair and its reconstruction gives both
    # |x - x'| <= 510 in unsigned 16-bit lanes; their squares sum exactly
    rng = np.random.default_rng(4)
    x = rng.integers(-255, 256, (2, 100_000))
    y = rng.integers(-255, 256, (2, 100_000))
    d = np.abs(x - y)
    word = (d[0] & 0xFFFF) | ((d[1] & 0xFFFF) << 16)
    got = (word & 0xFFFF) ** 2 + (word >> 16) ** 2
    assert np.array_equal(got, ((x - y) ** 2).sum(axis=0))


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
