"""The FP32 OpenMP CPU implementation that the benchmark times beside the GPU path (context only).

It computes the method in plain FP32, so near a bin edge its votes may fall in the neighbouring bin
(the bin coordinate n_phi (phi0 + pi) / 2 pi has a rounding error of a few 1e-4 bins at n_phi = 2048,
above the oracle's 1e-4 flag window); the checks are therefore statistical against the FP64 oracle,
plus exact properties of its own output."""
import numpy as np
import pytest

import baseline
import oracle
from paper_1310_7556_gb300 import eventgen as eg


@pytest.fixture(scope="module")
def small():
    w = eg.WORKLOADS["single_50trk"]
    ev = w.event(0)
    ref = oracle.run(w.geometry, w.binning, ev)
    cpu, M = baseline.run_event(baseline.make_binning(w.geometry, w.binning), ev, threads=4, want_accumulator=True)
    return w, ev, ref, cpu, M


def test_accumulator_agrees_with_the_oracle_but_for_edge_votes(small):
    w, ev, ref, cpu, M = small
    diff = M != ref["M"]
    assert diff.mean() < 1e-3
    # every differing cell is one where a vote moved by a bin: its mask is a subset of the
    # oracle's mask of the neighbouring cells on the same row, or the other way round
    R, P = M.shape
    for i, j in zip(*np.nonzero(diff)):
        around_ref = ref["M"][i, (j - 1) % P] | ref["M"][i, j] | ref["M"][i, (j + 1) % P]
        around_cpu = M[i, (j - 1) % P] | M[i, j] | M[i, (j + 1) % P]
        assert (M[i, j] & ~around_ref) == 0 or (ref["M"][i, j] & ~around_cpu) == 0


def test_candidates_and_confirmation_match_the_oracle_on_most_candidates(small):
    w, ev, ref, cpu, M = small
    oc = {(int(c["iq"]), int(c["jphi"])): q for q, c in enumerate(ref["candidates"])}
    cc = {(int(i), int(j)): q for q, (i, j) in enumerate(zip(cpu["iq"], cpu["jphi"]))}
    common = set(oc) & set(cc)
    assert len(common) >= 0.95 * len(oc) and len(common) >= 0.95 * len(cc)
    nmem = np.diff(ref["member_offsets"])
    agree = sum(1 for k in common if cpu["n_members"][cc[k]] == nmem[oc[k]]
                and (cpu["icot"][cc[k]], cpu["jz0"][cc[k]]) == (ref["stage2"]["icot"][oc[k]], ref["stage2"]["jz0"][oc[k]]))
    assert agree >= 0.9 * len(common)


def test_own_output_is_consistent(small):
    w, ev, ref, cpu, M = small
    # candidates in raster order, each a local maximum with at least `threshold` layers
    key = cpu["iq"].astype(np.int64) * w.binning.n_phi + cpu["jphi"]
    assert np.all(np.diff(key) > 0)
    counts = np.array([bin(int(m)).count("1") for m in cpu["mask"]])
    assert np.all(counts >= w.binning.threshold)
    assert np.all(cpu["mask"] == M[cpu["iq"], cpu["jphi"]])
    # the stage-2 mask holds only layers of the candidate's members; confirmation follows its size
    c2 = np.array([bin(int(m)).count("1") for m in cpu["mask2"]])
    assert np.all(cpu["confirmed"] == (c2 >= min(w.binning.threshold, w.geometry.n_layers)))


def test_thread_count_does_not_change_the_result(small):
    w, ev, ref, cpu, M = small
    b = baseline.make_binning(w.geometry, w.binning)
    for t in (1, 3):
        c2, M2 = baseline.run_event(b, ev, threads=t, want_accumulator=True)
        assert np.array_equal(M2, M)
        for f in baseline.FIELDS:
            assert np.array_equal(c2[f], cpu[f])
