"""The oracle against hand-worked values of the paper's own formulas (fixtures in tests/golden/,
each citing the passage it evaluates)."""
import os

import numpy as np

from oracle import baselines, wproj

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def test_eq5_baseline_index_hand_worked():
    rows = np.array(_rows("eq5_baseline_index_nant4.txt"), dtype=np.int64)
    got = baselines.baseline_index(rows[:, 0], rows[:, 1], 4)
    np.testing.assert_array_equal(got, rows[:, 2])
    assert sorted(set(got.tolist())) == list(range(baselines.n_baselines(4)))


def test_eq6_start_index_hand_worked():
    count, start = (np.array(r, dtype=np.int64) for r in _rows("eq6_start_index.txt"))
    n_ant = 3                                           # 6 baselines, autocorrelations included
    assert baselines.n_baselines(n_ant) == count.size
    bidx = np.repeat(np.arange(count.size), count)[::-1].copy()    # any row order
    c, s = baselines.baseline_starts(bidx, n_ant)
    np.testing.assert_array_equal(c, count)
    np.testing.assert_array_equal(s[:-1], start)
    assert s[-1] == count.sum()


def test_plane_supports_golden():
    for r in _rows("plane_supports.txt"):
        k = r.index(":")
        n_w, s_min, s_max = (int(x) for x in r[:k])
        expect = [int(x) for x in r[k + 1:]]
        assert wproj.plane_supports(n_w, s_min, s_max).tolist() == expect, r
