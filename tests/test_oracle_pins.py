"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle (or the shared event simulation) against a closed
form, an invariant of the method, a hand-derived case or a brute-force
computation in a different formulation -- never against a retyped copy of its
own formulas.  All run on the CPU.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1310_7556_gb300 import eventgen as eg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GEOM = eg.Geometry()


def _event(r, phi, z, layer):
    return eg.Event(np.asarray(r, np.float32), np.asarray(phi, np.float32), np.asarray(z, np.float32),
                    np.asarray(layer, np.uint8), np.zeros(len(r), np.int32))


def _centres(bn, i, j, m=None, n=None):
    k = bn.qpt_min + (i + 0.5) * (bn.qpt_max - bn.qpt_min) / bn.n_qpt
    phi0 = -math.pi + (j + 0.5) * 2.0 * math.pi / bn.n_phi
    cot = z0 = 0.0
    if m is not None:
        cot = bn.cot_min + (m + 0.5) * (bn.cot_max - bn.cot_min) / bn.n_cot
        z0 = bn.z0_min + (n + 0.5) * (bn.z0_max - bn.z0_min) / bn.n_z0
    return k, phi0, cot, z0


def _popcount(a):
    a = np.asarray(a, dtype=np.uint32)
    return np.unpackbits(a.view(np.uint8)).reshape(a.shape + (32,)).sum(-1)


# --------------------------------------------------------------------------------------------
# The event simulation, pinned to plane geometry (Sec. 4: tracks are circles in the transverse
# plane of a barrel detector).
# --------------------------------------------------------------------------------------------

def test_simulated_hits_lie_on_the_track_circle():
    """Noiseless hits sit on a circle of radius R = pT / (0.3 B) through the beam line whose
    tangent there points along phi0, and z advances with the arc length R * (subtended angle)."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        q = rng.choice([-1.0, 1.0])
        pt = math.exp(rng.uniform(math.log(0.5), math.log(100.0)))
        phi0, cot, z0 = rng.uniform(-math.pi, math.pi), rng.uniform(-6, 6), rng.normal(0, 5)
        r, phi, z, layer, _ = eg.helix_hits(GEOM, [q / pt], [phi0], [cot], [z0])
        R = 100.0 * pt / (0.3 * GEOM.b_tesla)                 # cm
        centre = q * R * np.array([-math.sin(phi0), math.cos(phi0)])
        pts = np.stack([r * np.cos(phi), r * np.sin(phi)], axis=1)
        assert np.allclose(np.linalg.norm(pts - centre, axis=1), R, rtol=1e-12, atol=1e-9)
        # every layer closer than the diameter is reached, no other
        assert sorted(layer.tolist()) == [l for l, rl in enumerate(GEOM.radii_cm) if rl <= 2 * R]
        # arc length from the subtended angle at the centre, computed with atan2
        a0 = np.arctan2(-centre[1], -centre[0])
        ah = np.arctan2(pts[:, 1] - centre[1], pts[:, 0] - centre[0])
        alpha = np.abs((ah - a0 + math.pi) % (2 * math.pi) - math.pi)
        assert np.allclose(z, z0 + cot * R * alpha, rtol=1e-10, atol=1e-9)


# --------------------------------------------------------------------------------------------
# Stage-1 vote
# --------------------------------------------------------------------------------------------

def test_golden_single_helix_fixtures():
    """Hand-derived worked examples (tests/golden/single_helix.json)."""
    with open(os.path.join(GOLDEN, "single_helix.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        bn = eg.Binning(**c["binning"])
        k, phi0, cot, z0 = _centres(bn, *c["generating_bin"], *c["generating_stage2_bin"])
        r, phi, z, layer, _ = eg.helix_hits(GEOM, [k], [phi0], [cot], [z0])
        b = oracle.make_binning(GEOM, bn)
        M, votes, flags = oracle.vote(b, _event(r, phi, z, layer))
        i, j = c["generating_bin"]
        assert int(M[i, j]) == c["expected_mask"]
        assert int(votes.sum()) == c["expected_votes"]
        cands = oracle.peaks(b, M)
        assert [(int(x["iq"]), int(x["jphi"]), int(x["mask"])) for x in cands] == \
            [tuple(x) for x in c["expected_candidates"]]


@pytest.mark.parametrize("seed", range(6))
def test_single_noiseless_helix_generating_bin_holds_all_layers(seed):
    """A noiseless helix with q/pT and phi0 on bin centres puts every reached layer in its own bin
    (closed form: the vote inverts the hit position exactly), and the peak search returns exactly
    one candidate: in the generating column, at the top of the run of rows of that column that hold
    every reached layer and contain the generating row (the first row of the q/pT plateau under the
    raster tie-break; one row above the generating one on the coarse grids, more on the paper's
    2048-row grid, where neighbouring rows shift the inner layers by a small part of a bin)."""
    rng = np.random.default_rng(100 + seed)
    for geom, bn in ((GEOM, eg.BINNING_SMALL), (GEOM, eg.BINNING_PILEUP), (GEOM, eg.BINNING_FINE),
                     (eg.PAPER_GEOMETRY, eg.BINNING_PAPER)):   # the last: the paper's detector and grid
        i = int(rng.integers(2, bn.n_qpt - 2))
        j = int(rng.integers(0, bn.n_phi))
        k, phi0, _, _ = _centres(bn, i, j)
        r, phi, z, layer, _ = eg.helix_hits(geom, [k], [phi0], [0.0], [0.0])
        b = oracle.make_binning(geom, bn)
        M, votes, flags = oracle.vote(b, _event(r, phi, z, layer))
        reached = sum(1 << int(l) for l in layer)
        assert int(M[i, j]) == reached
        assert not np.any(flags["row"] == i)      # votes at the generating row sit on bin centres
        if len(layer) >= bn.threshold:
            cands = oracle.peaks(b, M)
            assert len(cands) == 1
            top = i
            while top > 0 and int(M[top - 1, j]) == reached:
                top -= 1
            assert int(cands[0]["jphi"]) == j and int(cands[0]["iq"]) == top
            assert int(cands[0]["mask"]) == reached
            if bn is not eg.BINNING_PAPER:
                assert top in (i - 1, i)


def _exact_vote_count(b, r):
    """Number of q/pT bin centres k_i with |0.15 B (r/100) k_i| <= 1, by exact rational arithmetic."""
    c = Fraction(0.15) * Fraction(b.b_tesla) * Fraction(float(r)) / 100
    dk = (Fraction(b.qpt_max) - Fraction(b.qpt_min)) / b.n_qpt
    lim = 1 / c
    # i ranges over integers with -lim <= qpt_min + (i + 1/2) dk <= lim
    lo = math.ceil((-lim - Fraction(b.qpt_min)) / dk - Fraction(1, 2))
    hi = math.floor((lim - Fraction(b.qpt_min)) / dk - Fraction(1, 2))
    lo, hi = max(lo, 0), min(hi, b.n_qpt - 1)
    return max(0, hi - lo + 1)


@pytest.mark.parametrize("name", ["single_50trk", "pileup_100k", "paper_500"])
def test_vote_count_conservation(name):
    """Votes per layer equal the closed-form count of rows inside the |x| <= 1 domain (up to
    domain-flagged votes), and the masks never hold more layer bits than votes were cast."""
    w = eg.paper_workload(500) if name == "paper_500" else eg.WORKLOADS[name]
    ev = w.event(3)
    if ev.n_hits > 20000:
        ev = ev.subset(np.arange(20000))
    b = oracle.make_binning(w.geometry, w.binning)
    M, votes, flags = oracle.vote(b, ev)
    n_domain = int((flags["kind"] == 2).sum())
    for l in range(w.geometry.n_layers):
        radii = ev.r[ev.layer == l]
        uniq, cnt = np.unique(radii, return_counts=True)
        expect = sum(int(n) * _exact_vote_count(b, rr) for rr, n in zip(uniq, cnt))
        assert abs(int(votes[l]) - expect) <= n_domain
        assert int(((M >> l) & 1).sum()) <= int(votes[l])
    assert int(_popcount(M).sum()) <= int(votes.sum())


def test_cyclic_phi_rotation_shifts_accumulator():
    """Rotating every hit by m bin widths shifts the accumulator by m columns.  Bins may differ
    only where a vote of either event lies within the flag window of an edge (the FP32 inputs
    are rounded after rotation, moving votes by < 1e-4 bin)."""
    w = eg.WORKLOADS["single_50trk"]
    b = oracle.make_binning(w.geometry, w.binning)
    ev = w.event(1)
    M, _, fl = oracle.vote(b, ev)
    for m in (1, 37, -5, w.binning.n_phi // 2):
        rot = (ev.phi.astype(np.float64) + m * 2.0 * math.pi / b.n_phi)
        rot = np.mod(rot + math.pi, 2 * math.pi) - math.pi
        ev2 = eg.Event(ev.r, rot.astype(np.float32), ev.z, ev.layer, ev.track)
        M2, _, fl2 = oracle.vote(b, ev2)
        shifted = np.roll(M, m, axis=1)
        diff = np.argwhere(shifted != M2)
        allowed = set()
        for f in fl:
            for jj in (f["bin"], f["alt"]):
                if jj >= 0:
                    allowed.add((int(f["row"]), int((jj + m) % b.n_phi)))
        for f in fl2:
            for jj in (f["bin"], f["alt"]):
                if jj >= 0:
                    allowed.add((int(f["row"]), int(jj)))
        assert all((int(i), int(j)) in allowed for i, j in diff)
        assert len(diff) <= len(fl) + len(fl2)
        # candidates rotate with the accumulator where their neighbourhood is untouched by flags
        c1 = {(int(c["iq"]), int((c["jphi"] + m) % b.n_phi)) for c in oracle.peaks(b, M)}
        c2 = {(int(c["iq"]), int(c["jphi"])) for c in oracle.peaks(b, M2)}
        near = {(i + di, (j + dj) % b.n_phi) for (i, j) in allowed for di in (-1, 0, 1) for dj in (-1, 0, 1)}
        assert {c for c in c1 ^ c2 if c not in near} == set()


def _brute_force_votes(b, r, phi, layer, mp):
    """Bin-major brute force with a different predicate: bin (i, j) receives hit h when
    f(d) = sin(d) - x changes sign across the bin, d = phi - phi0 on the branch |d| <= pi/2
    where f increases; evaluated at 40 significant digits.  No arcsine is used."""
    mp.mp.dps = 40
    M = np.zeros((b.n_qpt, b.n_phi), np.uint16)
    two_pi = 2 * mp.pi
    w = two_pi / b.n_phi
    half_pi = mp.pi / 2
    dk = (mp.mpf(b.qpt_max) - mp.mpf(b.qpt_min)) / b.n_qpt
    for h in range(len(r)):
        rr, ph = mp.mpf(float(r[h])), mp.mpf(float(phi[h]))
        for i in range(b.n_qpt):
            k = mp.mpf(b.qpt_min) + (i + mp.mpf(1) / 2) * dk
            x = mp.mpf(15) / 100 * mp.mpf(b.b_tesla) * rr / 100 * k
            if abs(x) > 1:
                continue
            for j in range(b.n_phi):
                edge = -mp.pi + j * w
                hi = ph - edge
                hi = hi - two_pi * mp.floor((hi + mp.pi) / two_pi)     # into [-pi, pi)
                lo = hi - w
                if hi < -half_pi or lo >= half_pi:
                    continue
                ok_lo = lo < -half_pi or mp.sin(lo) < x      # the root lies above lo
                ok_hi = hi >= half_pi or mp.sin(hi) >= x     # ... and not above hi
                if ok_lo and ok_hi:
                    M[i, j] |= 1 << int(layer[h])
    return M


@pytest.mark.parametrize("seed", range(3))
def test_vote_matches_brute_force_sign_change(seed):
    """Tiny random events: the oracle's hit-major FP64 vote equals a bin-major high-precision
    sign-change search, except at votes the oracle flags as edge votes."""
    mp = pytest.importorskip("mpmath")
    rng = np.random.default_rng(seed)
    bn = eg.Binning(n_qpt=24, qpt_min=-2.0, qpt_max=2.0, n_phi=48, threshold=3)
    b = oracle.make_binning(GEOM, bn)
    n = 12
    layer = rng.integers(0, 10, n).astype(np.uint8)
    r = np.asarray(GEOM.radii_cm, np.float32)[layer]
    phi = rng.uniform(-math.pi, math.pi, n).astype(np.float32)
    M, _, flags = oracle.vote(b, _event(r, phi, np.zeros(n), layer))
    Mb = _brute_force_votes(b, r, phi, layer, mp)
    diff = np.argwhere(M != Mb)
    allowed = {(int(f["row"]), int(jj)) for f in flags for jj in (f["bin"], f["alt"]) if jj >= 0}
    assert all((int(i), int(j)) in allowed for i, j in diff)


def test_vote_matches_high_precision_arithmetic():
    """Every unflagged FP64 vote lands in the bin of the exact (40-digit) computation."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rng = np.random.default_rng(11)
    bn = eg.BINNING_FINE
    b = oracle.make_binning(GEOM, bn)
    n = 6
    layer = rng.integers(0, 10, n).astype(np.uint8)
    r = np.asarray(GEOM.radii_cm, np.float32)[layer]
    phi = rng.uniform(-math.pi, math.pi, n).astype(np.float32)
    M, _, flags = oracle.vote(b, _event(r, phi, np.zeros(n), layer))
    flagged = {(int(f["hit"]), int(f["row"])) for f in flags}
    dk = (mp.mpf(bn.qpt_max) - mp.mpf(bn.qpt_min)) / bn.n_qpt
    checked = 0
    for h in range(n):
        for i in range(0, bn.n_qpt, 7):
            k = mp.mpf(bn.qpt_min) + (i + mp.mpf(1) / 2) * dk
            x = mp.mpf(15) / 100 * mp.mpf(GEOM.b_tesla) * mp.mpf(float(r[h])) / 100 * k
            if abs(x) > 1 or (h, i) in flagged:
                continue
            u = bn.n_phi * (mp.mpf(float(phi[h])) - mp.asin(x) + mp.pi) / (2 * mp.pi)
            j = int(mp.floor(u)) % bn.n_phi
            assert (int(M[i, j]) >> int(layer[h])) & 1
            checked += 1
    assert checked > 200


def test_missing_layers_tolerated():
    """The Hough transform tolerates missing hits (Sec. 4): removing up to L - k layers of a
    noiseless helix keeps one candidate at the generating column, holding the remaining layers."""
    bn = eg.BINNING_SMALL
    b = oracle.make_binning(GEOM, bn)
    i, j = 70, 33
    k, phi0, _, _ = _centres(bn, i, j)
    r, phi, z, layer, _ = eg.helix_hits(GEOM, [k], [phi0], [0.0], [0.0])
    rng = np.random.default_rng(5)
    for drop in range(0, GEOM.n_layers - bn.threshold + 1):
        keep = np.sort(rng.permutation(len(r))[drop:])
        M, _, _ = oracle.vote(b, _event(r[keep], phi[keep], z[keep], layer[keep]))
        cands = oracle.peaks(b, M)
        assert len(cands) == 1 and int(cands[0]["jphi"]) == j
        assert int(cands[0]["mask"]) == sum(1 << int(l) for l in layer[keep])
    keep = np.arange(bn.threshold - 1)
    M, _, _ = oracle.vote(b, _event(r[keep], phi[keep], z[keep], layer[keep]))
    assert len(oracle.peaks(b, M)) == 0


# --------------------------------------------------------------------------------------------
# Peak search: hand-derived accumulators (tests/golden/peak_cases.json)
# --------------------------------------------------------------------------------------------

def test_golden_peak_cases():
    with open(os.path.join(GOLDEN, "peak_cases.json")) as f:
        spec = json.load(f)
    for case in spec["cases"]:
        nq, nphi = case["shape"]
        M = np.zeros((nq, nphi), np.uint16)
        for i, j, mask in case["cells"]:
            M[i, j] = mask
        bn = eg.Binning(n_qpt=nq, qpt_min=-1, qpt_max=1, n_phi=nphi, threshold=case["threshold"])
        got = [(int(c["iq"]), int(c["jphi"])) for c in oracle.peaks(oracle.make_binning(GEOM, bn), M)]
        assert got == [tuple(x) for x in case["expected"]], case["name"]


def test_peaks_invariants_on_random_accumulators():
    """Candidates are never 8-neighbours of one another, each reaches the threshold and dominates
    its 3 x 3 block, and every strict maximum of its 3 x 3 block above threshold is found."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        nq, nphi = 9, 16
        M = rng.integers(0, 1 << 6, (nq, nphi)).astype(np.uint16)
        bn = eg.Binning(n_qpt=nq, qpt_min=-1, qpt_max=1, n_phi=nphi, threshold=3)
        cands = {(int(c["iq"]), int(c["jphi"])) for c in oracle.peaks(oracle.make_binning(GEOM, bn), M)}
        p = _popcount(M)
        padded = np.zeros((nq + 2, nphi), int)
        padded[1:-1] = p
        for i in range(nq):
            for j in range(nphi):
                block = [padded[i + 1 + di, (j + dj) % nphi] for di in (-1, 0, 1) for dj in (-1, 0, 1)
                         if (di, dj) != (0, 0)]
                strict = p[i, j] >= 3 and all(v < p[i, j] for v in block)
                if strict:
                    assert (i, j) in cands
                if (i, j) in cands:
                    assert p[i, j] >= 3 and all(v <= p[i, j] for v in block)
        for (i, j) in cands:
            for di in (-1, 0, 1):
                for dj in (-1, 0, 1):
                    if (di, dj) != (0, 0):
                        assert (i + di, (j + dj) % nphi) not in cands


# --------------------------------------------------------------------------------------------
# The count accumulator (Sec. 8: A[B[i]] += 1): a cell holds its number of votes
# --------------------------------------------------------------------------------------------

def _counts_binning(geometry, binning, **kw):
    return oracle.make_binning(geometry, eg.Binning(**{**binning.__dict__, "accumulator": eg.ACC_COUNTS, **kw}))


def test_golden_count_peak_cases():
    """Hand-derived cases (tests/golden/count_peak_cases.json), each read both ways: as counts and
    as layer masks, which disagree on every case but one."""
    with open(os.path.join(GOLDEN, "count_peak_cases.json")) as f:
        spec = json.load(f)
    for case in spec["cases"]:
        nq, nphi = case["shape"]
        M = np.zeros((nq, nphi), np.uint16)
        for i, j, v in case["cells"]:
            M[i, j] = v
        for acc, key in ((eg.ACC_COUNTS, "expected"), (eg.ACC_LAYERS, "expected_layers")):
            bn = eg.Binning(n_qpt=nq, qpt_min=-1, qpt_max=1, n_phi=nphi, threshold=case["threshold"],
                            accumulator=acc)
            got = [(int(c["iq"]), int(c["jphi"]), int(c["mask"])) for c in oracle.peaks(oracle.make_binning(GEOM, bn), M)]
            assert [(i, j) for i, j, _ in got] == [tuple(x) for x in case[key]], (case["name"], key)
            assert all(v == int(M[i, j]) for i, j, v in got)   # the candidate carries the cell's value


def test_count_peaks_are_the_strict_maxima_of_distinct_counts():
    """With every count distinct there are no ties, so the candidates are exactly the cells at or
    above threshold that equal the maximum of their 3 x 3 block -- computed here with
    scipy.ndimage.maximum_filter (phi0 wrapped, rows outside the grid empty)."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(11)
    for nq, nphi, thr in ((9, 16, 1), (17, 64, 900), (33, 128, 3000)):
        M = (rng.permutation(nq * nphi) + 1).astype(np.uint16).reshape(nq, nphi)
        padded = np.zeros((nq + 2, nphi + 2), np.int64)
        padded[1:-1, 1:-1] = M
        padded[1:-1, 0] = M[:, -1]
        padded[1:-1, -1] = M[:, 0]
        local_max = ndimage.maximum_filter(padded, size=3, mode="constant", cval=0)[1:-1, 1:-1]
        expect = [(int(i), int(j)) for i, j in np.argwhere((M == local_max) & (M >= thr))]
        bn = eg.Binning(n_qpt=nq, qpt_min=-1, qpt_max=1, n_phi=nphi, threshold=thr, accumulator=eg.ACC_COUNTS)
        got = [(int(c["iq"]), int(c["jphi"])) for c in oracle.peaks(oracle.make_binning(GEOM, bn), M)]
        assert got == expect and len(got) > 0


def test_counts_are_sums_of_single_hit_votes():
    """A cell's count is the number of hits whose vote fell in it: summing, over the hits one at a
    time, the cells each single hit marks in the (pinned) layer accumulator gives the count
    accumulator of the whole event, cell for cell."""
    w = eg.WORKLOADS["single_50trk"]
    ev = w.event(4).subset(np.arange(60))
    bl = oracle.make_binning(w.geometry, w.binning)
    bc = _counts_binning(w.geometry, w.binning)
    expect = np.zeros((bl.n_qpt, bl.n_phi), np.int64)
    for h in range(ev.n_hits):
        Mh, _, _ = oracle.vote(bl, ev.subset(np.array([h])))
        expect += Mh != 0
    Mc, votes, _ = oracle.vote(bc, ev)
    assert np.array_equal(Mc.astype(np.int64), expect)
    assert int(Mc.sum()) == int(votes.sum())


@pytest.mark.parametrize("name", ["single_50trk", "pileup_100k", "paper_500"])
def test_counts_conserve_votes_and_bound_the_layer_masks(name):
    """Unsaturated counts sum to the votes cast; a cell is non-empty in one accumulator exactly
    when it is in the other, and its count is at least its number of layers."""
    w = eg.paper_workload(500) if name == "paper_500" else eg.WORKLOADS[name]
    ev = w.event(1)
    if ev.n_hits > 20000:
        ev = ev.subset(np.arange(20000))
    Ml, vl, fl = oracle.vote(oracle.make_binning(w.geometry, w.binning), ev)
    Mc, vc, fc = oracle.vote(_counts_binning(w.geometry, w.binning), ev)
    assert np.array_equal(vl, vc) and np.array_equal(fl, fc)
    assert int(Mc.max()) < 65535 and int(Mc.sum()) == int(vc.sum())
    assert np.array_equal(Mc > 0, Ml != 0)
    assert np.all(Mc >= _popcount(Ml))


def test_counts_equal_layer_counts_for_one_hit_per_layer():
    """A single track leaves at most one hit per layer, so no two votes in a cell share a layer:
    every count equals the number of layers in the same cell's mask."""
    rng = np.random.default_rng(21)
    for geom, bn in ((GEOM, eg.BINNING_SMALL), (GEOM, eg.BINNING_PILEUP), (eg.PAPER_GEOMETRY, eg.BINNING_PAPER)):
        i, j = int(rng.integers(2, bn.n_qpt - 2)), int(rng.integers(0, bn.n_phi))
        k, phi0, _, _ = _centres(bn, i, j)
        r, phi, z, layer, _ = eg.helix_hits(geom, [k], [phi0], [0.0], [0.0])
        ev = _event(r, phi, z, layer)
        Ml, _, _ = oracle.vote(oracle.make_binning(geom, bn), ev)
        Mc, _, _ = oracle.vote(_counts_binning(geom, bn), ev)
        assert np.array_equal(Mc.astype(np.int64), _popcount(Ml))
        assert int(Mc[i, j]) == len(layer)


def test_duplicated_hits_multiply_counts():
    """Every hit taken d times: each count is d times the original, the layer masks do not change."""
    w = eg.WORKLOADS["single_50trk"]
    ev = w.event(6)
    d = 3
    dup = ev.subset(np.repeat(np.arange(ev.n_hits), d))
    bl, bc = oracle.make_binning(w.geometry, w.binning), _counts_binning(w.geometry, w.binning)
    Mc1, _, _ = oracle.vote(bc, ev)
    Mcd, _, _ = oracle.vote(bc, dup)
    assert np.array_equal(Mcd.astype(np.int64), d * Mc1.astype(np.int64))
    assert np.array_equal(oracle.vote(bl, dup)[0], oracle.vote(bl, ev)[0])


def test_counts_saturate_at_65535():
    """70,000 copies of one hit: every cell it votes in holds 65535, the votes are all counted."""
    bn = eg.Binning(n_qpt=2, qpt_min=-0.5, qpt_max=0.5, n_phi=64, threshold=1, accumulator=eg.ACC_COUNTS)
    n = 70000
    ev = _event(np.full(n, 30.0), np.full(n, 0.3), np.zeros(n), np.zeros(n, np.uint8))
    M, votes, _ = oracle.vote(oracle.make_binning(GEOM, bn), ev)
    assert int(votes.sum()) == 2 * n
    assert sorted(M[M > 0].tolist()) == [65535, 65535] and np.count_nonzero(M[0]) == 1


def test_unknown_accumulator_kind_is_rejected():
    bn = eg.Binning(n_qpt=4, qpt_min=-1, qpt_max=1, n_phi=64, threshold=1, accumulator=2)
    with pytest.raises(ValueError):
        oracle.vote(oracle.make_binning(GEOM, bn), _event([30.0], [0.1], [0.0], [0]))


# --------------------------------------------------------------------------------------------
# Non-prompt tracks: the impact-parameter axis d0
# --------------------------------------------------------------------------------------------

BINNING_D0 = eg.Binning(n_qpt=128, qpt_min=-1.0, qpt_max=1.0, n_phi=256, threshold=8,
                        n_d0=9, d0_min=-0.9, d0_max=0.9)


def _d0_centre(bn, m):
    return bn.d0_min + (m + 0.5) * (bn.d0_max - bn.d0_min) / bn.n_d0


def test_displaced_hits_lie_on_the_track_circle():
    """Plane geometry of the displaced forward model: every hit is on the circle of radius
    R = 100 / (0.3 B |k|) about the centre (d0 + R_signed)(-sin phi0, cos phi0), the circle's
    closest approach to the beam line is |d0| away, z advances with the arc length from it (from the
    chord, 2 R asin(chord / 2R), not the swept angle the model uses), and with d0 = 0 the model
    reproduces the prompt helices."""
    rng = np.random.default_rng(31)
    k = rng.uniform(-1.2, 1.2, 40)
    phi0 = rng.uniform(-math.pi, math.pi, 40)
    d0 = rng.uniform(-2.0, 2.0, 40)
    cot = rng.uniform(-2.0, 2.0, 40)
    z0 = rng.uniform(-5.0, 5.0, 40)
    r, phi, z, layer, tk = eg.displaced_hits(GEOM, k, phi0, d0, cot, z0)
    assert len(r) > 200
    rs = 100.0 / (0.3 * GEOM.b_tesla * k)
    n = np.stack([-np.sin(phi0), np.cos(phi0)], 1)
    centre = (d0 + rs)[:, None] * n
    assert np.allclose(np.abs(np.linalg.norm(centre, axis=1) - np.abs(rs)), np.abs(d0), atol=1e-9)
    pts = np.stack([r * np.cos(phi), r * np.sin(phi)], 1)
    assert np.allclose(np.linalg.norm(pts - centre[tk], axis=1), np.abs(rs[tk]), rtol=1e-10, atol=1e-8)
    chord = np.linalg.norm(pts - (d0[:, None] * n)[tk], axis=1)
    arc = 2.0 * np.abs(rs[tk]) * np.arcsin(np.clip(chord / (2.0 * np.abs(rs[tk])), -1.0, 1.0))
    assert np.allclose(z, z0[tk] + cot[tk] * arc, rtol=1e-9, atol=1e-7)
    prompt = eg.helix_hits(GEOM, k, phi0, cot, z0)
    zero = eg.displaced_hits(GEOM, k, phi0, np.zeros(40), cot, z0)
    for a, b in zip(prompt, zero):
        assert np.allclose(np.asarray(a, float), np.asarray(b, float), rtol=0, atol=1e-11)


@pytest.mark.parametrize("seed", range(4))
def test_displaced_helix_generating_cell_holds_all_layers(seed):
    """A noiseless displaced helix with q/pT, phi0 and d0 on bin centres puts every reached layer
    in its generating (d0, q/pT, phi0) cell, no vote of that row is flagged, and the raster-first
    cell holding every reached layer is a candidate."""
    rng = np.random.default_rng(200 + seed)
    bn = BINNING_D0
    b = oracle.make_binning(GEOM, bn)
    for _ in range(4):
        i, j, m = int(rng.integers(2, bn.n_qpt - 2)), int(rng.integers(0, bn.n_phi)), int(rng.integers(0, bn.n_d0))
        k, phi0, _, _ = _centres(bn, i, j)
        r, phi, z, layer, _ = eg.displaced_hits(GEOM, [k], [phi0], [_d0_centre(bn, m)], [0.0], [0.0])
        M, votes, flags = oracle.vote(b, _event(r, phi, z, layer))
        assert M.shape == (bn.n_d0 * bn.n_qpt, bn.n_phi)
        reached = sum(1 << int(l) for l in layer)
        row = m * bn.n_qpt + i
        assert int(M[row, j]) == reached
        assert not np.any(flags["row"] == row)
        cands = oracle.peaks(b, M)
        first = np.argwhere(M == reached)[0]
        got = {(int(c["id0"]) * bn.n_qpt + int(c["iq"]), int(c["jphi"])) for c in cands}
        assert (int(first[0]), int(first[1])) in got
        assert all(int(c["mask"]) != 0 for c in cands)


def test_d0_vote_matches_plane_geometry():
    """The d0 vote of each (hit, q/pT row, d0 slice) against plane geometry: the forward model puts
    a track of phi0 = 0 through the hit's layer at azimuth D(k, d0, r), so by rotation the track
    through the hit has phi0 = phi - D; its bin must be the oracle's (votes the oracle flags
    excepted), and where the forward model finds no crossing the oracle casts no vote."""
    rng = np.random.default_rng(41)
    # q/pT up to 3 and |d0| up to 6 cm: many (row, layer) pairs have no crossing (|x| > 1, |d0| > r)
    bn = eg.Binning(n_qpt=32, qpt_min=-3.0, qpt_max=3.0, n_phi=512, threshold=8, n_d0=7, d0_min=-7.0, d0_max=7.0)
    b = oracle.make_binning(GEOM, bn)
    checked = missing = 0
    for _ in range(60):
        l = int(rng.integers(0, GEOM.n_layers))
        phi = float(rng.uniform(-math.pi, math.pi))
        ev = _event([GEOM.radii_cm[l]], [phi], [0.0], [l])
        M, _, flags = oracle.vote(b, ev)
        flagged = {int(f["row"]) for f in flags}
        one = eg.Geometry(radii_cm=(GEOM.radii_cm[l],), b_tesla=GEOM.b_tesla)
        for row in range(b.n_rows):
            if row in flagged:
                continue
            m, i = divmod(row, bn.n_qpt)
            k, _, _, _ = _centres(bn, i, 0)
            rr, ph, _, _, _ = eg.displaced_hits(one, [k], [0.0], [_d0_centre(bn, m)], [0.0], [0.0])
            voted = np.nonzero(M[row])[0]
            if len(rr) == 0:
                assert len(voted) == 0, (row, voted)
                missing += 1
                continue
            phi0 = np.float64(np.float32(phi)) - ph[0]
            j = int(math.floor(bn.n_phi * (phi0 + math.pi) / (2 * math.pi))) % bn.n_phi
            assert voted.tolist() == [j], (row, voted, j)
            checked += 1
    assert checked > 5000 and missing > 100


def test_centred_d0_slice_equals_the_prompt_grid():
    """With an odd number of d0 bins centred on 0 the middle slice has d0 = 0 exactly and must be
    the prompt accumulator, cell for cell, with the same flags."""
    w = eg.WORKLOADS["single_50trk"]
    ev = w.event(3)
    prompt = oracle.make_binning(w.geometry, w.binning)
    b3 = oracle.make_binning(w.geometry, eg.Binning(**{**w.binning.__dict__, "n_d0": 3, "d0_min": -1.5, "d0_max": 1.5}))
    Mp, vp, fp = oracle.vote(prompt, ev)
    M3, v3, f3 = oracle.vote(b3, ev)
    q = w.binning.n_qpt
    assert np.array_equal(M3[q:2 * q], Mp)
    mid = f3[(f3["row"] >= q) & (f3["row"] < 2 * q)].copy()
    mid["row"] -= q
    assert np.array_equal(mid, fp)
    assert int(v3.sum()) >= int(vp.sum())


def test_single_d0_slice_at_zero_is_the_prompt_oracle():
    """One d0 bin centred on 0: the d0 grid is the prompt grid, and the 3x3x3 rule with no
    neighbouring slices is the 3x3 rule -- same accumulator, flags, candidates and stage 2."""
    w = eg.WORKLOADS["single_50trk"]
    ev = w.event(1)
    prompt = oracle.run(w.geometry, w.binning, ev)
    one = oracle.run(w.geometry, eg.Binning(**{**w.binning.__dict__, "n_d0": 1, "d0_min": -0.5, "d0_max": 0.5}), ev)
    for k in ("M", "vote_flags", "candidates", "member_offsets", "members", "stage2"):
        assert np.array_equal(one[k], prompt[k]), k


def test_golden_peak3_cases():
    with open(os.path.join(GOLDEN, "peak3_cases.json")) as f:
        spec = json.load(f)
    for case in spec["cases"]:
        nd, nq, nphi = case["shape"]
        M = np.zeros((nd * nq, nphi), np.uint16)
        for m, i, j, mask in case["cells"]:
            M[m * nq + i, j] = mask
        bn = eg.Binning(n_qpt=nq, qpt_min=-1, qpt_max=1, n_phi=nphi, threshold=case["threshold"],
                        n_d0=nd, d0_min=-1.0, d0_max=1.0)
        got = [(int(c["id0"]), int(c["iq"]), int(c["jphi"])) for c in oracle.peaks(oracle.make_binning(GEOM, bn), M)]
        assert got == [tuple(x) for x in case["expected"]], case["name"]


def test_peaks3_are_the_strict_maxima_of_distinct_values():
    """Distinct counts in a d0 grid: the candidates are exactly the cells at or above threshold equal
    to the maximum of their 3 x 3 x 3 block (scipy.ndimage.maximum_filter; phi0 wrapped, rows and
    slices outside the grid empty)."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(13)
    nd, nq, nphi = 5, 9, 64
    vals = (rng.permutation(nd * nq * nphi) + 1).astype(np.uint16).reshape(nd, nq, nphi)
    padded = np.zeros((nd + 2, nq + 2, nphi + 2), np.int64)
    padded[1:-1, 1:-1, 1:-1] = vals
    padded[1:-1, 1:-1, 0] = vals[:, :, -1]
    padded[1:-1, 1:-1, -1] = vals[:, :, 0]
    local_max = ndimage.maximum_filter(padded, size=3, mode="constant", cval=0)[1:-1, 1:-1, 1:-1]
    expect = [tuple(int(v) for v in x) for x in np.argwhere((vals == local_max) & (vals >= 500))]
    bn = eg.Binning(n_qpt=nq, qpt_min=-1, qpt_max=1, n_phi=nphi, threshold=500, accumulator=eg.ACC_COUNTS,
                    n_d0=nd, d0_min=-1.0, d0_max=1.0)
    got = [(int(c["id0"]), int(c["iq"]), int(c["jphi"]))
           for c in oracle.peaks(oracle.make_binning(GEOM, bn), vals.reshape(nd * nq, nphi))]
    assert got == expect and len(got) > 20


def test_stage2_displaced_helix_closed_form():
    """Member hits of a noiseless displaced helix with cot(theta) and z0 on stage-2 bin centres all
    vote for the generating (cot, z0) cell: the arc length from the closest approach is the one
    the forward model advanced z by."""
    bn = eg.Binning(**{**eg.BINNING_PILEUP.__dict__, "n_d0": 8, "d0_min": -2.0, "d0_max": 2.0})
    b = oracle.make_binning(GEOM, bn)
    rng = np.random.default_rng(19)
    for _ in range(8):
        i, j = int(rng.integers(0, bn.n_qpt)), int(rng.integers(0, bn.n_phi))
        m, n, md = int(rng.integers(0, bn.n_cot)), int(rng.integers(0, bn.n_z0)), int(rng.integers(0, bn.n_d0))
        k, phi0, cot, z0 = _centres(bn, i, j, m, n)
        r, phi, z, layer, _ = eg.displaced_hits(GEOM, [k], [phi0], [_d0_centre(bn, md)], [cot], [z0])
        ev = _event(r, phi, z, layer)
        cand = np.zeros(1, oracle.CAND_DTYPE)
        cand["iq"], cand["jphi"], cand["id0"] = i, j, md
        res, _ = oracle.stage2(b, ev, cand, np.array([0, len(r)], np.int64), np.arange(len(r), dtype=np.int64))
        assert (int(res[0]["icot"]), int(res[0]["jz0"])) == (m, n)
        assert int(res[0]["mask2"]) == sum(1 << int(l) for l in layer)


def test_d0_members_reproduce_candidate_masks():
    """In a d0 grid, the members of each candidate (hits whose vote on its q/pT row of its d0 slice
    fell in its column) OR to its mask."""
    w = eg.displaced_workload()
    b = oracle.make_binning(w.geometry, w.binning)
    ev = w.event(0)
    M, _, _ = oracle.vote(b, ev)
    cands = oracle.peaks(b, M)
    offsets, mem, _ = oracle.members(b, ev, cands)
    assert len(cands) > 20 and len(np.unique(cands["id0"])) > 3
    for q, c in enumerate(cands):
        acc = 0
        for h in mem[offsets[q]:offsets[q + 1]]:
            acc |= 1 << int(ev.layer[h])
        assert acc == int(c["mask"])


# --------------------------------------------------------------------------------------------
# Membership and the second-stage vote
# --------------------------------------------------------------------------------------------

def test_member_layers_reproduce_candidate_mask():
    """A cell's mask is the OR of the layer bits of the hits that voted into it, so the members
    found by re-deriving the votes must OR to exactly the candidate's mask."""
    w = eg.WORKLOADS["single_50trk"]
    b = oracle.make_binning(w.geometry, w.binning)
    ev = w.event(2)
    M, _, _ = oracle.vote(b, ev)
    cands = oracle.peaks(b, M)
    offsets, mem, _ = oracle.members(b, ev, cands)
    assert len(cands) > 10
    for q, c in enumerate(cands):
        hits = mem[offsets[q]:offsets[q + 1]]
        assert np.all(np.diff(hits) > 0)
        acc = 0
        for h in hits:
            acc |= 1 << int(ev.layer[h])
        assert acc == int(c["mask"])


def test_stage2_single_helix_closed_form():
    """Member hits of a noiseless helix with cot(theta) and z0 on stage-2 bin centres all vote for
    the generating (cot, z0) cell, which is then the stage-2 maximum with every layer."""
    bn = eg.BINNING_PILEUP
    b = oracle.make_binning(GEOM, bn)
    rng = np.random.default_rng(9)
    for _ in range(8):
        i, j = int(rng.integers(0, bn.n_qpt)), int(rng.integers(0, bn.n_phi))
        m, n = int(rng.integers(0, bn.n_cot)), int(rng.integers(0, bn.n_z0))
        k, phi0, cot, z0 = _centres(bn, i, j, m, n)
        r, phi, z, layer, _ = eg.helix_hits(GEOM, [k], [phi0], [cot], [z0])
        ev = _event(r, phi, z, layer)
        cand = np.zeros(1, oracle.CAND_DTYPE)
        cand["iq"], cand["jphi"] = i, j
        offsets = np.array([0, len(r)], np.int64)
        res, _ = oracle.stage2(b, ev, cand, offsets, np.arange(len(r), dtype=np.int64))
        assert (int(res[0]["icot"]), int(res[0]["jz0"])) == (m, n)
        assert int(res[0]["mask2"]) == sum(1 << int(l) for l in layer)
        assert int(res[0]["n_votes"]) <= len(r) * bn.n_cot


def test_stage2_matches_geometric_brute_force():
    """Stage-2 cells from a separate computation: z0 from the arc length R * alpha, alpha the
    angle the chord subtends at the circle's centre (atan2 geometry, no arcsine)."""
    w = eg.WORKLOADS["single_50trk"]
    bn = w.binning
    b = oracle.make_binning(w.geometry, bn)
    ev = w.event(4)
    M, _, _ = oracle.vote(b, ev)
    cands = oracle.peaks(b, M)[:12]
    offsets, mem, _ = oracle.members(b, ev, cands)
    res, zflags = oracle.stage2(b, ev, cands, offsets, mem)
    flagged = {int(f["cand"]) for f in zflags}
    dt = (bn.cot_max - bn.cot_min) / bn.n_cot
    for q, c in enumerate(cands):
        if q in flagged:
            continue
        k = bn.qpt_min + (int(c["iq"]) + 0.5) * (bn.qpt_max - bn.qpt_min) / bn.n_qpt
        R = 100.0 / (0.3 * w.geometry.b_tesla * abs(k))          # cm
        M2 = np.zeros((bn.n_cot, bn.n_z0), np.uint16)
        for h in mem[offsets[q]:offsets[q + 1]]:
            rr = float(ev.r[h])
            # chord of length rr from the beam line; the centre sits at distance R from both ends
            half = rr / 2.0
            alpha = 2.0 * math.atan2(half, math.sqrt(max(R * R - half * half, 0.0)))
            s = R * alpha
            for m in range(bn.n_cot):
                t = bn.cot_min + (m + 0.5) * dt
                u = bn.n_z0 * (float(ev.z[h]) - s * t - bn.z0_min) / (bn.z0_max - bn.z0_min)
                if 0 <= u < bn.n_z0:
                    M2[m, int(math.floor(u))] |= 1 << int(ev.layer[h])
        p = _popcount(M2)
        best = int(np.argmax(p))
        assert (int(res[q]["icot"]), int(res[q]["jz0"])) == divmod(best, bn.n_z0)
        assert int(res[q]["mask2"]) == int(M2.flat[best])
