"""The parity rule itself, on the CPU: a mistake planted in the oracle's own accumulator is caught,
a legitimate move of a flagged vote is not."""
import numpy as np
import pytest

import oracle
from paper_1310_7556_gb300 import eventgen as eg

from parity import assert_accumulator_parity, assert_count_parity


def _counts_case():
    w = eg.with_binning(eg.WORKLOADS["single_50trk"], accumulator=eg.ACC_COUNTS)
    ev = w.event(0)
    M, _, flags = oracle.vote(oracle.make_binning(w.geometry, w.binning), ev)
    return M, flags


def test_count_rule_accepts_the_oracle_itself():
    M, flags = _counts_case()
    assert assert_count_parity(M, M, flags) == 0


def test_count_rule_catches_an_extra_vote_at_an_unflagged_cell():
    M, flags = _counts_case()
    touched = {(int(f["row"]), int(b)) for f in flags for b in (f["bin"], f["alt"]) if b >= 0}
    i, j = next((int(i), int(j)) for i, j in np.argwhere(M > 0) if (int(i), int(j)) not in touched)
    bad = M.copy()
    bad[i, j] += 1
    with pytest.raises(AssertionError):
        assert_count_parity(bad, M, flags)


def test_count_rule_accepts_a_flagged_vote_moved_to_its_other_bin():
    M, flags = _counts_case()
    f = next(f for f in flags if int(f["kind"]) == 1 and f["bin"] >= 0 and f["alt"] >= 0)
    moved = M.copy()
    moved[int(f["row"]), int(f["bin"])] -= 1
    moved[int(f["row"]), int(f["alt"])] += 1
    assert assert_count_parity(moved, M, flags) == 2


def test_layer_rule_catches_a_dropped_layer_bit():
    w = eg.WORKLOADS["single_50trk"]
    M, _, flags = oracle.vote(oracle.make_binning(w.geometry, w.binning), w.event(0))
    touched = {(int(f["row"]), int(b)) for f in flags for b in (f["bin"], f["alt"]) if b >= 0}
    i, j = next((int(i), int(j)) for i, j in np.argwhere(M > 0) if (int(i), int(j)) not in touched)
    bad = M.copy()
    bad[i, j] &= bad[i, j] - 1   # drop the lowest layer bit
    with pytest.raises(AssertionError):
        assert_accumulator_parity(bad, M, flags)
