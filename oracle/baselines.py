"""Baseline grouping of the paper's GPU gridding scheme (Sec. 2.2) -- TEST INFRASTRUCTURE.

The paper groups visibilities by baseline, time-ordered within each, before gridding, so that
one thread per support tap can walk a baseline's samples and keep its sum in a register while
the grid point stays the same. Three steps, each here in its plainest form:

  baseline_index : Eq. 5, the index of the baseline (I_ant1, I_ant2) from the antenna IDs;
  baseline_starts: Eq. 6, the start of every baseline's range as the exclusive prefix sum of
                   the per-baseline sample counts C;
  baseline_order : the rows placed baseline by baseline at those starts, each baseline's rows
                   in their original (time) order -- a counting sort.

Pinned in tests/test_oracle_baselines.py against the enumeration of the upper triangle of the
antenna-pair matrix (numpy.triu_indices), brute-force counts and Python's sorted() on
(baseline, row) pairs.
"""
from __future__ import annotations

import numpy as np


def n_baselines(n_ant: int) -> int:
    """Number of Eq. 5 indices: antenna pairs with I_ant1 <= I_ant2, autocorrelations included."""
    return n_ant * (n_ant + 1) // 2


def baseline_index(ant1, ant2, n_ant: int) -> np.ndarray:
    """Eq. 5: I_B = (-S^2 + 2 S N_ant + S) / 2 + |I_ant1 - I_ant2| with S = min(I_ant1, I_ant2).

    Integer arithmetic throughout (-S^2 + 2 S N + S = S (2N - S + 1) is always even)."""
    a1 = np.asarray(ant1, dtype=np.int64)
    a2 = np.asarray(ant2, dtype=np.int64)
    s = np.minimum(a1, a2)
    num = -s * s + 2 * s * n_ant + s
    assert np.all(num % 2 == 0)
    return num // 2 + np.abs(a1 - a2)


def baseline_starts(bidx: np.ndarray, n_ant: int) -> tuple[np.ndarray, np.ndarray]:
    """Eq. 6: (C, start) with C[b] the number of rows of baseline b and
    start[b] = C[0] + ... + C[b-1]; start has one more entry, the row total."""
    nb = n_baselines(n_ant)
    count = np.zeros(nb, dtype=np.int64)
    for b in np.asarray(bidx, dtype=np.int64):
        count[b] += 1
    start = np.zeros(nb + 1, dtype=np.int64)
    for b in range(nb):
        start[b + 1] = start[b] + count[b]
    return count, start


def baseline_order(bidx: np.ndarray, n_ant: int) -> np.ndarray:
    """Row indices grouped by baseline (rising I_B), rows of one baseline in rising row order:
    each row, taken in row order, goes to the next free slot of its baseline's range."""
    _, start = baseline_starts(bidx, n_ant)
    cursor = start[:-1].copy()
    perm = np.empty(len(bidx), dtype=np.int64)
    for r, b in enumerate(np.asarray(bidx, dtype=np.int64)):
        perm[cursor[b]] = r
        cursor[b] += 1
    return perm
