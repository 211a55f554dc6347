"""Greedy angle-minimising row search of §3 (Eq. (5)-(6), Fig. 1 abmApprox).

TEST INFRASTRUCTURE (CPU oracle; never imported by the product path).

For a row order wp and a search space D = P^8 (§3.2), the rows of the exact
DCT are approximated one at a time, in the order wp:

    t_{wp(k)} = argmin_{d in D} angle(c_{wp(k)}, d)
                subject to <d, t_{wp(i)}> = 0 for every row already chosen.

Readings taken where the paper is silent or inconsistent
---------------------------------------------------------
* Orthogonality is pairwise with every row already chosen (§3.4 and the
  constraint under Eq. (6)).  The listing in Fig. 1 tests that the *sum* of
  the inner products is zero, which would admit non-orthogonal rows; the text
  governs.
* The zero vector is not a candidate (its angle is undefined).
* When no candidate is orthogonal to the rows already chosen, the order
  fails (``None``).  The listing would silently write the first element of D.
* Minimising the angle is maximising cos = <c, d> / ||d|| (||c|| = 1), which
  avoids arccos; values within ``TIE_TOL`` of the best are exact ties in real
  arithmetic (they arise for d and 2d, and for rows 3 and 7 over D1), and the
  ``tie`` policy decides: "small" keeps the smaller-norm vector, "large" the
  larger-norm one.  Remaining ties (same norm) keep the lexicographically
  smallest vector of the enumeration in ``search_space``.
* §4.1 fixes rows 1 and 5 to the all-ones vector and (1,-1,-1,1,1,-1,-1,1)
  and searches the 6! = 720 orders of the remaining six rows.
"""
from __future__ import annotations

import itertools
from functools import lru_cache

import numpy as np

from .matrices import dct_matrix

TIE_TOL = 1e-12
P1 = (0, 1, -1)
P2 = (0, 1, -1, 2, -2)
ROW1 = np.ones(8, dtype=np.int64)
ROW5 = np.array([1, -1, -1, 1, 1, -1, -1, 1], dtype=np.int64)


@lru_cache(maxsize=None)
def search_space(P: tuple) -> np.ndarray:
    """All of P^8 except the zero vector, as an (|P|^8 - 1, 8) int64 array."""
    vals = np.array(sorted(P), dtype=np.int64)
    grid = np.stack(np.meshgrid(*([vals] * 8), indexing="ij"), axis=-1).reshape(-1, 8)
    keep = np.any(grid != 0, axis=1)
    return np.ascontiguousarray(grid[keep])


class _Space:
    """Candidate set with per-row cosines and norms, computed once."""

    def __init__(self, P: tuple):
        self.D = search_space(P)
        self.norm2 = np.einsum("ij,ij->i", self.D, self.D)
        C = dct_matrix(8)
        # cos(c_k, d) = <c_k, d> / ||d||, rows of C have unit norm.
        self.cos = (self.D.astype(np.float64) @ C.T) / np.sqrt(self.norm2)[:, None]
        self._orth = {}

    def orth_mask(self, t: np.ndarray) -> np.ndarray:
        key = tuple(int(v) for v in t)
        m = self._orth.get(key)
        if m is None:
            m = (self.D @ np.asarray(t, dtype=np.int64)) == 0
            self._orth[key] = m
        return m

    def pick(self, k: int, allowed: np.ndarray, tie: str):
        """Index of the best candidate for exact row k (0-based) or None."""
        if not allowed.any():
            return None
        cos = np.where(allowed, self.cos[:, k], -np.inf)
        best = cos.max()
        ties = np.nonzero(allowed & (cos >= best - TIE_TOL))[0]
        if len(ties) == 1:
            return int(ties[0])
        n2 = self.norm2[ties]
        target = n2.min() if tie == "small" else n2.max()
        ties = ties[n2 == target]
        return int(ties[0])


_SPACES: dict = {}


def _space(P: tuple) -> _Space:
    if P not in _SPACES:
        _SPACES[P] = _Space(P)
    return _SPACES[P]


def abm_approx(order, P: tuple = P2, tie: str = "small", fixed=None):
    """Run the greedy search for one row order (1-based row numbers).

    ``fixed`` maps 1-based row numbers to preset rows (e.g. {1: ROW1, 5: ROW5});
    preset rows constrain orthogonality but are not searched.  Returns the
    8x8 int64 matrix T, or None when the order dead-ends.
    """
    sp = _space(P)
    T = np.zeros((8, 8), dtype=np.int64)
    allowed = np.ones(len(sp.D), dtype=bool)
    for row, vec in (fixed or {}).items():
        T[row - 1] = vec
        allowed &= sp.orth_mask(vec)
    for row in order:
        idx = sp.pick(row - 1, allowed, tie)
        if idx is None:
            return None
        T[row - 1] = sp.D[idx]
        allowed &= sp.orth_mask(sp.D[idx])
    return T


def search_all_orders(P: tuple = P2, tie: str = "small"):
    """§4.1: rows 1 and 5 fixed, all 720 orders of rows {2,3,4,6,7,8}.

    Returns a list of (order, T or None).  The permutation tree is walked
    depth first so that shared prefixes are evaluated once; the result for
    each order is identical to ``abm_approx(order, P, tie, fixed)``.
    """
    sp = _space(P)
    rows = (2, 3, 4, 6, 7, 8)
    base = np.ones(len(sp.D), dtype=bool) & sp.orth_mask(ROW1) & sp.orth_mask(ROW5)
    out = []

    def walk(prefix, remaining, allowed, chosen):
        if not remaining:
            T = np.zeros((8, 8), dtype=np.int64)
            T[0], T[4] = ROW1, ROW5
            for r, v in chosen.items():
                T[r - 1] = v
            out.append((tuple(prefix), T))
            return
        for r in remaining:
            idx = sp.pick(r - 1, allowed, tie)
            rest = tuple(x for x in remaining if x != r)
            if idx is None:
                # dead end: every completion of this prefix fails
                for tail in itertools.permutations(rest):
                    out.append((tuple(prefix) + (r,) + tail, None))
                continue
            v = sp.D[idx]
            walk(prefix + [r], rest, allowed & sp.orth_mask(v), {**chosen, r: v})

    walk([], rows, base, {})
    out.sort(key=lambda x: x[0])
    return out


# ---- the same search for any blocklength N ---------------------------------------
#
# §6.2 extends the question to N = 16 (search space P^16, 3^16 candidates for
# P = {-1, 0, 1}) and times one fixed row sequence.  ``abm_approx_n`` is the
# search above written for any N and any alphabet, with the same readings
# (pairwise orthogonality, zero vector excluded, cosines in FP64 with the
# TIE_TOL tolerance, the norm policy, then the enumeration order).  Candidates
# are enumerated as base-|P| numbers over sorted(P), first coordinate most
# significant: the order of ``search_space``.  Plain vectorised evaluation in
# chunks; no pruning.

def candidate_block(P: tuple, N: int, start: int, stop: int) -> np.ndarray:
    """Candidates start..stop-1 of the full enumeration of P^N (zero vector
    included), as an int8 array of shape (stop - start, N)."""
    vals = np.array(sorted(P), dtype=np.int8)
    idx = np.arange(start, stop, dtype=np.int64)
    base = len(vals)
    out = np.empty((stop - start, N), dtype=np.int8)
    for pos in range(N - 1, -1, -1):
        out[:, pos] = vals[idx % base]
        idx //= base
    return out


def abm_approx_n(N: int, order, P: tuple, tie: str = "small", fixed=None,
                 chunk: int = 1 << 22, partial: bool = False):
    """Greedy search for blocklength N over P^N for the row order ``order``
    (0-based rows of the N-point DCT), with ``fixed`` = {row: vector} preset.
    Returns the N x N int64 matrix (rows not in ``order`` or ``fixed`` stay
    zero), or None when a row has no orthogonal candidate left.  With
    ``partial`` it returns (T, complete) instead: on a dead end T holds the
    rows chosen before it and complete is False.

    The candidates still allowed (nonzero, orthogonal to every preset and to
    every row chosen so far) are kept as one boolean per candidate and
    narrowed by each new row before the next row's cosines are taken, as in
    the 8-point search above.  The candidate vectors are enumerated once per
    call (int8, in chunks)."""
    C = dct_matrix(N)
    total = len(P) ** N
    T = np.zeros((N, N), dtype=np.int64)
    blocks = [(s, candidate_block(P, N, s, min(total, s + chunk)))
              for s in range(0, total, chunk)]
    allowed = np.ones(total, dtype=bool)
    pending = []  # rows whose orthogonality is not yet applied to `allowed`
    for row, vec in (fixed or {}).items():
        T[row] = vec
        pending.append(np.asarray(vec, dtype=np.int64))
    for row in order:
        best_cos, best_idx, best_n2 = [], [], []
        for s, Db in blocks:
            idx = np.nonzero(allowed[s:s + len(Db)])[0]
            D = Db[idx].astype(np.int64)
            keep = np.einsum("ij,ij->i", D, D) > 0
            for t in pending:
                keep &= (D @ t) == 0
            allowed[s + idx[~keep]] = False
            idx, D = idx[keep], D[keep]
            n2 = np.einsum("ij,ij->i", D, D)
            best_cos.append((D.astype(np.float64) @ C[row]) / np.sqrt(n2))
            best_idx.append(s + idx)
            best_n2.append(n2)
        pending = []
        cos_all = np.concatenate(best_cos)
        if cos_all.size == 0:
            return (T, False) if partial else None
        idx_all = np.concatenate(best_idx)
        n2_all = np.concatenate(best_n2)
        best = cos_all.max()
        sel = np.nonzero(cos_all >= best - TIE_TOL)[0]
        if len(sel) > 1:
            n2 = n2_all[sel]
            sel = sel[n2 == (n2.min() if tie == "small" else n2.max())]
        first = int(idx_all[sel].min())  # the first tied candidate of the enumeration
        v = candidate_block(P, N, first, first + 1)[0].astype(np.int64)
        T[row] = v
        pending.append(v)
    return (T, True) if partial else T
