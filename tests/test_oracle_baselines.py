"""Pins for the oracle's baseline grouping (Sec. 2.2, Eq. 5 and Eq. 6). CPU only."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("n_ant", [1, 2, 3, 7, 27, 128])
def test_eq5_enumerates_the_upper_triangle(n_ant):
    """Eq. 5 numbers the pairs (S, S + d), d >= 0, row by row: the position of the pair in
    numpy's row-major upper-triangle enumeration (diagonal included). So it is a bijection
    onto [0, N_ant (N_ant + 1) / 2)."""
    i, j = np.triu_indices(n_ant)
    b = oracle.baseline_index(i, j, n_ant)
    np.testing.assert_array_equal(b, np.arange(len(i)))
    assert len(i) == oracle.n_baselines(n_ant)


def test_eq5_is_symmetric_in_the_antennas():
    rng = np.random.default_rng(3)
    a1, a2 = rng.integers(0, 40, 500), rng.integers(0, 40, 500)
    np.testing.assert_array_equal(oracle.baseline_index(a1, a2, 40), oracle.baseline_index(a2, a1, 40))


def test_eq5_worked_values():
    """Hand-worked: N_ant = 4, pairs (0,0) -> 0, (0,3) -> 3, (1,1) -> 4, (1,3) -> 6, (2,3) -> 8,
    (3,3) -> 9: S = 1 gives (-1 + 8 + 1) / 2 = 4, S = 2 gives (-4 + 16 + 2) / 2 = 7."""
    a1 = np.array([0, 0, 1, 3, 2, 3])
    a2 = np.array([0, 3, 1, 1, 3, 3])
    np.testing.assert_array_equal(oracle.baseline_index(a1, a2, 4), [0, 3, 4, 6, 8, 9])


def test_eq6_starts_and_order_brute_force():
    rng = np.random.default_rng(4)
    n_ant, nrow = 9, 400
    a1, a2 = rng.integers(0, n_ant, nrow), rng.integers(0, n_ant, nrow)
    b = oracle.baseline_index(a1, a2, n_ant)
    count, start = oracle.baseline_starts(b, n_ant)
    for k in range(oracle.n_baselines(n_ant)):
        assert count[k] == int(np.sum(b == k))
        assert start[k] == int(np.sum(b < k))
    assert start[-1] == nrow
    perm = oracle.baseline_order(b, n_ant)
    want = [r for _, r in sorted((int(b[r]), r) for r in range(nrow))]
    np.testing.assert_array_equal(perm, want)


def test_synthetic_rows_have_n_time_samples_per_cross_baseline():
    """The time-major synthetic rows: every cross baseline has n_time rows, every
    autocorrelation none, and ordering puts row t * N_bl + k at start[k'] + t."""
    n_ant, n_time = 6, 5
    a1, a2 = synth.row_antennas(n_ant, n_time)
    b = oracle.baseline_index(a1, a2, n_ant)
    count, start = oracle.baseline_starts(b, n_ant)
    auto = oracle.baseline_index(np.arange(n_ant), np.arange(n_ant), n_ant)
    assert np.all(count[auto] == 0)
    cross = np.setdiff1d(np.arange(oracle.n_baselines(n_ant)), auto)
    assert np.all(count[cross] == n_time)
    perm = oracle.baseline_order(b, n_ant)
    nbl = n_ant * (n_ant - 1) // 2
    for k in range(nbl):
        rows = perm[start[b[k]]:start[b[k] + 1]]
        np.testing.assert_array_equal(rows, k + nbl * np.arange(n_time))
