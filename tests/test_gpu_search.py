"""GPU greedy angle search (tdct_search) against the CPU oracle: every row
order of §4.1 over D1 and D2 with both tie policies, the extended alphabets
listed in §4.1, and the longer blocklengths of §6.2 (N = 12, 16 with
P = {-1, 0, 1})."""
import numpy as np
import pytest

import paper_1808_02950_gb300 as P
from oracle import search as S

pytestmark = pytest.mark.gpu
FIXED = {0: tuple(S.ROW1), 4: tuple(S.ROW5)}


@pytest.mark.parametrize("alph", [S.P1, S.P2])
@pytest.mark.parametrize("tie", ["small", "large"])
def test_search_all_720_orders_of_section_4_1(alph, tie):
    want = dict(S.search_all_orders(alph, tie))
    for order, T in want.items():
        got, complete = P.tdct_search(8, alph, [o - 1 for o in order], FIXED, tie)
        if T is None:
            assert not complete, order
        else:
            assert complete and np.array_equal(np.array(got), T), order


@pytest.mark.parametrize("alph", [(0, 1, -1, 4, -4), (0, 1, -1, 8, -8), (0, 1, -1, 2, -2, 4, -4),
                                  (0, 2, -2, 4, -4, 8, -8)])
def test_search_extended_alphabets(alph):
    rng = np.random.default_rng(len(alph))
    for _ in range(2):
        order = [int(v) for v in rng.permutation([1, 2, 3, 5, 6, 7])]
        want = S.abm_approx_n(8, order, alph, "small", {0: S.ROW1, 4: S.ROW5})
        got, complete = P.tdct_search(8, alph, order, FIXED, "small")
        assert (want is None and not complete) or (complete and np.array_equal(np.array(got), want))


def test_search_N12_natural_order():
    want = S.abm_approx_n(12, range(12), S.P1, "small")
    got, complete = P.tdct_search(12, S.P1, range(12), None, "small")
    assert (want is None and not complete) or (complete and np.array_equal(np.array(got), want))


@pytest.mark.slow
def test_search_N16_P1():
    """§6.2's case (3^16 - 1 candidates per row, natural row order): every row
    the GPU finds equals the oracle's, and both dead-end at the same row with
    the same rows before it (the oracle's full search takes about 20 s on one
    host core)."""
    got, complete = P.tdct_search(16, S.P1, range(16), None, "small")
    want, want_complete = S.abm_approx_n(16, range(16), S.P1, "small", partial=True)
    G = np.array(got, dtype=np.int64)
    assert complete == want_complete
    assert np.array_equal(G, want)
    found = np.count_nonzero(np.abs(want).sum(axis=1))
    assert found >= 6  # several rows beyond the presets are compared
    gram = G @ G.T
    assert np.count_nonzero(gram - np.diag(np.diag(gram))) == 0


@pytest.mark.parametrize("cap", [0, 1, 3])
@pytest.mark.parametrize("tie", ["small", "large"])
def test_search_hit_list_overflow_rescans(cap, tie):
    """A row whose screened candidates overflow the hit list is decided by a
    second full scan; with tiny capacities (D2 has many exact ties: scaled
    copies of a vector) every such row takes that path, and the results still
    match the oracle."""
    want = dict(S.search_all_orders(S.P2, tie))
    orders = list(want)[::37]
    try:
        P.tdct_debug_search_hit_cap(cap)
        for order in orders:
            got, complete = P.tdct_search(8, S.P2, [o - 1 for o in order], FIXED, tie)
            T = want[order]
            if T is None:
                assert not complete, order
            else:
                assert complete and np.array_equal(np.array(got), T), order
    finally:
        P.tdct_debug_search_hit_cap(-1)
