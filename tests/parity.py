"""Comparison of the CUDA path with the FP64 oracle under the parity rule.

Rule: the integer layer masks and the candidate list are bit-exact, except where a vote the
oracle flags (its bin coordinate within 1e-4 bin of an edge, or |x| within 1e-6 of 1) may
legitimately land on the other side in FP32; the number of mismatched (cell, layer) pairs must
not exceed the number of flagged votes, and each must be explained by one.  Counts likewise:
each cell equal up to the flagged votes that may have left it or landed in it.
"""
from __future__ import annotations

import numpy as np


def _allowed_cells(flags, n_phi):
    """(row, bin, layer) triples a flagged vote may touch; a domain-edge flag with no bin on the
    oracle side allows any bin of the row for that layer (stored with bin -1)."""
    allowed = set()
    for f in flags:
        row, lay = int(f["row"]), int(f["layer"])
        for b in (f["bin"], f["alt"]):
            if b >= 0:
                allowed.add((row, int(b) % n_phi, lay))
        if int(f["kind"]) == 2:
            allowed.add((row, -1, lay))
    return allowed


def accumulator_mismatches(M_gpu: np.ndarray, M_ref: np.ndarray, flags) -> tuple[list, list]:
    """Returns (all mismatched (i, j, layer) triples, those no flagged vote explains)."""
    n_phi = M_ref.shape[1]
    allowed = _allowed_cells(flags, n_phi)
    diff = np.argwhere(M_gpu != M_ref)
    mism, unexplained = [], []
    for i, j in diff:
        x = int(M_gpu[i, j]) ^ int(M_ref[i, j])
        for l in range(16):
            if (x >> l) & 1:
                t = (int(i), int(j), l)
                mism.append(t)
                if t not in allowed and (int(i), -1, l) not in allowed:
                    unexplained.append(t)
    return mism, unexplained


def count_slack(flags, shape):
    """Per cell, how far a count may fall below (lo <= 0) or rise above (hi >= 0) the oracle's:
    a flagged vote may leave its oracle bin and land in its alternative bin; a domain-edge flag
    with no oracle bin may add one vote anywhere on its row (row_extra)."""
    n_q, n_phi = shape
    lo = np.zeros(shape, np.int64)
    hi = np.zeros(shape, np.int64)
    row_extra = np.zeros(n_q, np.int64)
    for f in flags:
        row, b, a = int(f["row"]), int(f["bin"]), int(f["alt"])
        if b >= 0:
            lo[row, b % n_phi] -= 1
        if a >= 0:
            hi[row, a % n_phi] += 1
        if int(f["kind"]) == 2 and b < 0:
            row_extra[row] += 1
    return lo, hi, row_extra


def assert_count_parity(M_gpu, M_ref, flags):
    """Count accumulator: every cell equal, except for the flagged votes' moves; returns the number
    of cells that differ."""
    lo, hi, row_extra = count_slack(flags, M_ref.shape)
    diff = M_gpu.astype(np.int64) - M_ref.astype(np.int64)
    bad = np.argwhere((diff < lo) | (diff > hi + row_extra[:, None]))
    assert len(bad) == 0, f"{len(bad)} counts differ beyond the flagged votes: " + \
        str([(int(i), int(j), int(M_gpu[i, j]), int(M_ref[i, j])) for i, j in bad[:8]])
    assert int(np.abs(diff).sum()) <= 2 * len(flags)
    return int(np.count_nonzero(diff))


def assert_accumulator_parity(M_gpu, M_ref, flags, counts=False):
    if counts:
        return assert_count_parity(M_gpu, M_ref, flags)
    mism, unexplained = accumulator_mismatches(M_gpu, M_ref, flags)
    assert not unexplained, f"{len(unexplained)} accumulator bits differ at unflagged votes: {unexplained[:8]}"
    assert len(mism) <= len(flags), f"{len(mism)} mismatched bits > {len(flags)} flagged votes"
    return len(mism)


def _touched(flags, n_phi):
    cells = set()
    for f in flags:
        for b in (f["bin"], f["alt"]):
            if b >= 0:
                cells.add((int(f["row"]), int(b) % n_phi))
        if int(f["kind"]) == 2:
            cells.add((int(f["row"]), -1))
    return cells


def stacked(cands, n_qpt):
    """Oracle candidates with iq as the stacked row id0 * n_qpt + iq, as the GPU reports them."""
    out = cands.copy()
    out["iq"] = cands["id0"] * n_qpt + cands["iq"]
    return out


def assert_candidate_parity(c_gpu, c_ref, flags, n_phi, q_rows=None):
    """Candidate lists equal, except candidates whose 3 x 3 block (3 x 3 x 3 with a d0 axis of
    q_rows rows per slice; rows stacked) holds a cell a flagged vote touched."""
    touched = _touched(flags, n_phi)
    rows_any = {i for (i, j) in touched if j == -1}

    def neighbour_rows(i):
        if q_rows is None:
            return [i - 1, i, i + 1]
        m, q = divmod(i, q_rows)
        return [(m + dm) * q_rows + q + di for dm in (-1, 0, 1) for di in (-1, 0, 1) if 0 <= q + di < q_rows]

    def near(i, j):
        for ii in neighbour_rows(i):
            if ii in rows_any:
                return True
            for dj in (-1, 0, 1):
                if (ii, (j + dj) % n_phi) in touched:
                    return True
        return False

    g = {(int(c["iq"]), int(c["jphi"])): int(c["mask"]) for c in c_gpu}
    r = {(int(c["iq"]), int(c["jphi"])): int(c["mask"]) for c in c_ref}
    bad = [k for k in set(g) ^ set(r) if not near(*k)]
    bad += [k for k in set(g) & set(r) if g[k] != r[k] and not near(*k)]
    assert not bad, f"{len(bad)} candidates differ away from flagged votes: {sorted(bad)[:8]}"
    # order: raster
    keys = [(int(c["iq"]), int(c["jphi"])) for c in c_gpu]
    assert keys == sorted(keys), "GPU candidates are not in raster order"
    return len(set(g) ^ set(r))


def assert_members_and_stage2_parity(c_gpu, off_gpu, mem_gpu, ref, threshold, n_layers=16, counts=False):
    """Member lists and stage-2 results of candidates present on both sides.

    A member list may differ only by hits whose vote on that row the oracle flags; a stage-2
    result may differ only for such candidates or where the oracle flags a z0 vote.  A candidate is
    confirmed when its stage-2 cell holds min(threshold, n_layers) layers.  With the count
    accumulator every candidate's member count equals its count (below saturation)."""
    confirm = min(threshold, n_layers)
    if counts:
        for c in c_gpu:
            if int(c["mask"]) < 65535 and not int(c["flags"]) & 2:
                assert int(c["n_members"]) == int(c["mask"]), f"({int(c['iq'])}, {int(c['jphi'])}): members vs count"
    c_ref = ref["candidates"]
    n_qpt = ref.get("n_qpt", 0)
    index_ref = {(int(c["id0"]) * n_qpt + int(c["iq"]), int(c["jphi"])): q for q, c in enumerate(c_ref)}
    mflag_hits = {}
    for f in ref["member_flags"]:
        mflag_hits.setdefault(int(f["cand"]), set()).add(int(f["hit"]))
    zflag_cands = {int(f["cand"]) for f in ref["stage2_flags"]}
    checked = 0
    for q, c in enumerate(c_gpu):
        key = (int(c["iq"]), int(c["jphi"]))
        if key not in index_ref:
            continue
        p = index_ref[key]
        mg = set(mem_gpu[off_gpu[q]:off_gpu[q + 1]].tolist())
        mr = set(ref["members"][ref["member_offsets"][p]:ref["member_offsets"][p + 1]].tolist())
        assert list(mem_gpu[off_gpu[q]:off_gpu[q + 1]]) == sorted(mg), "member list not sorted"
        diff = mg ^ mr
        assert diff <= mflag_hits.get(p, set()), f"candidate {key}: members differ at unflagged hits {sorted(diff)[:8]}"
        assert int(c["n_members"]) == len(mg)
        if diff or p in zflag_cands:
            continue
        s = ref["stage2"][p]
        assert (int(c["icot"]), int(c["jz0"]), int(c["mask2"])) == (int(s["icot"]), int(s["jz0"]), int(s["mask2"])), \
            f"candidate {key}: stage 2 {(int(c['icot']), int(c['jz0']), int(c['mask2']))} vs oracle {tuple(int(v) for v in s)[:3]}"
        assert (int(c["flags"]) & 1) == (1 if bin(int(s["mask2"])).count("1") >= confirm else 0)
        checked += 1
    return checked
