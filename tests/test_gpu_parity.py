"""Parity of the CUDA path with the FP64 oracle, called through the C ABI (needs a GPU).

Element by element: the accumulator's layer masks, the vote count, the candidate list (raster
order), member lists and stage-2 results, bit-exact except where the oracle flags a vote within
its edge window (see tests/parity.py for the rule)."""
import math

import numpy as np
import pytest

import oracle
from paper_1310_7556_gb300 import eventgen as eg

from parity import (assert_accumulator_parity, assert_candidate_parity,
                    assert_members_and_stage2_parity, stacked)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1310_7556_gb300 import binding as b
    b.load()
    return b


def run_gpu(binding, geometry, binning, ev, tiling=None, where="host", max_candidates=1 << 18):
    with binding.HoughContext(geometry, binning, max_hits=max(ev.n_hits, 1), max_candidates=max_candidates) as ctx:
        if tiling:
            ctx.set_tiling(**tiling) if isinstance(tiling, dict) else ctx.set_tiling(*tiling)
        if where == "host":
            ctx.vote_event(ev)
        else:
            import torch
            t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (ev.r, ev.phi, ev.z, ev.layer)]
            torch.cuda.synchronize()
            ctx.vote(*t, n_hits=ev.n_hits, where=binding.DEVICE)
        ctx.peaks()
        ctx.stage2()
        M = ctx.accumulator()
        cands = ctx.candidates()
        st = ctx.stats()
        off, mem = ctx.members(len(cands))
    return dict(M=M, candidates=cands, stats=st, member_offsets=off, members=mem)


def check_event(binding, geometry, binning, ev, **kw):
    ref = oracle.run(geometry, binning, ev)
    ref["n_qpt"] = binning.n_qpt
    d0 = binning.n_d0 > 0
    got = run_gpu(binding, geometry, binning, ev, **kw)
    counts = binning.accumulator == eg.ACC_COUNTS
    n_bits = assert_accumulator_parity(got["M"], ref["M"], ref["vote_flags"], counts=counts)
    assert int(got["stats"].votes) == int(ref["votes_by_layer"].sum())
    for l in range(geometry.n_layers):
        assert int(got["stats"].votes_by_layer[l]) == int(ref["votes_by_layer"][l])
    n_c = assert_candidate_parity(got["candidates"], stacked(ref["candidates"], binning.n_qpt), ref["vote_flags"],
                                  binning.n_phi, q_rows=binning.n_qpt if d0 else None)
    checked = assert_members_and_stage2_parity(got["candidates"], got["member_offsets"], got["members"], ref,
                                               binning.threshold, geometry.n_layers, counts)
    return dict(ref=ref, got=got, mismatched_bits=n_bits, mismatched_cands=n_c, stage2_checked=checked)


@pytest.mark.parametrize("index", range(4))
def test_single_event_50_tracks(binding, index):
    w = eg.WORKLOADS["single_50trk"]
    r = check_event(binding, w.geometry, w.binning, w.event(index))
    assert r["stage2_checked"] > 0


def test_pileup_event_full_size(binding):
    """The 100k-hit pileup event at its full 512 x 2048 binning, every cell compared."""
    w = eg.WORKLOADS["pileup_100k"]
    r = check_event(binding, w.geometry, w.binning, w.event(0))
    assert r["got"]["stats"].uniform_layers == (1 << 10) - 1
    assert r["got"]["stats"].refined_votes == 0


@pytest.mark.parametrize("n_tracks", [100, 5000])
def test_paper_geometry_2048_grid(binding, n_tracks):
    """The paper's detector (ten layers evenly spaced to 110 cm, 0.4 mm resolution, transverse
    plane) on its 2048 x 2048 grid, at a small and at the largest event of its timing sweep."""
    w = eg.paper_workload(n_tracks)
    r = check_event(binding, w.geometry, w.binning, w.event(0))
    assert r["got"]["stats"].uniform_layers == (1 << 10) - 1


def test_fine_binning_event_full_size(binding):
    """The 400k-hit, 1024 x 4096 event, every cell compared."""
    w = eg.WORKLOADS["fine_4m"]
    check_event(binding, w.geometry, w.binning, w.event(0))


def test_device_pointers_match_host_path(binding):
    w = eg.WORKLOADS["pileup_100k"]
    ev = w.event(5).subset(np.arange(30000))
    a = run_gpu(binding, w.geometry, w.binning, ev, where="host")
    b = run_gpu(binding, w.geometry, w.binning, ev, where="device")
    assert np.array_equal(a["M"], b["M"])
    assert np.array_equal(a["candidates"], b["candidates"])


@pytest.mark.parametrize("tiling", [(1, 64, 128, 1), (7, 128, 256, 1), (16, 256, 256, 1), (32, 512, 512, 1),
                                    (64, 1024, 1024, 1), (3, 2048, 128, 1), (16, 256, 256, 0, 1),
                                    (16, 256, 256, 0, 3), (16, 256, 256, 0, 8), (16, 256, 256, 0, 16),
                                    (16, 256, 256, 1, 5), (16, 256, 256, 0, 1, 1, 64, 256),
                                    (16, 256, 256, 0, 1, 3, 128, 512), (16, 256, 256, 0, 1, 5, 512, 1024),
                                    (16, 256, 256, 0, 2, 7, 256, 256), (16, 256, 256, 0, 1, 8, 2048, 512),
                                    (16, 256, 256, 0, 1, 16, 256, 512), (16, 256, 256, 0, 4, 32, 128, 256)])
def test_tilings_agree_bit_for_bit(binding, tiling):
    """Every tile shape of the scatter kernel (ragged last slabs: 512 rows by 7 or 3), every band
    height of the peak search, and every gather tile (rows x columns x threads; ragged last row
    bands; a full-row tile whose profile windows exceed their shared-memory slot and are read from
    global memory) gives the same result."""
    w = eg.WORKLOADS["pileup_100k"]
    ev = w.event(2).subset(np.arange(40000))
    base = run_gpu(binding, w.geometry, w.binning, ev)
    other = run_gpu(binding, w.geometry, w.binning, ev, tiling=tiling)
    assert np.array_equal(base["M"], other["M"])
    assert np.array_equal(base["candidates"], other["candidates"])


def test_per_vote_path_for_non_uniform_radii(binding):
    """Hits of a layer at different radii take the FP32 asinf path with FP64 edge refinement."""
    w = eg.WORKLOADS["pileup_100k"]
    ev = w.event(3).subset(np.arange(20000))
    rng = np.random.default_rng(1)
    ev.r = (ev.r + rng.uniform(-0.5, 0.5, ev.n_hits)).astype(np.float32)
    r = check_event(binding, w.geometry, w.binning, ev)
    st = r["got"]["stats"]
    assert st.uniform_layers == 0 and st.general_votes == st.votes and st.refined_votes > 0


def test_mixed_uniform_and_non_uniform_layers(binding):
    w = eg.WORKLOADS["single_50trk"]
    ev = w.event(7)
    jitter = ev.layer % 2 == 1
    ev.r = np.where(jitter, ev.r * np.float32(1.003), ev.r).astype(np.float32)
    ev.r[np.nonzero(jitter)[0][::2]] *= np.float32(0.999)
    r = check_event(binding, w.geometry, w.binning, ev)
    assert r["got"]["stats"].uniform_layers == 0b0101010101


# ---------------------------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------------------------

def _event(r, phi, z, layer):
    return eg.Event(np.asarray(r, np.float32), np.asarray(phi, np.float32), np.asarray(z, np.float32),
                    np.asarray(layer, np.uint8), np.zeros(len(r), np.int32))


def test_empty_event(binding):
    w = eg.WORKLOADS["single_50trk"]
    got = run_gpu(binding, w.geometry, w.binning, _event([], [], [], []))
    assert not got["M"].any() and len(got["candidates"]) == 0 and got["stats"].votes == 0


def test_single_hit_and_extreme_azimuths(binding):
    w = eg.WORKLOADS["pileup_100k"]
    pi32 = np.float32(math.pi)
    phis = [0.0, pi32, -pi32, np.nextafter(pi32, np.float32(0)), 3.1415926, -3.1415926, 999.0, -999.0, 1e-30]
    for phi in phis:
        check_event(binding, w.geometry, w.binning, _event([110.0], [phi], [0.0], [9]))


def test_all_hits_at_one_azimuth(binding):
    """Degenerate pileup: every hit of every layer at the same phi (hot-spot atomics, one bucket)."""
    w = eg.WORKLOADS["pileup_100k"]
    n = 5000
    layer = np.arange(n) % 10
    r = np.asarray(w.geometry.radii_cm, np.float32)[layer]
    check_event(binding, w.geometry, w.binning, _event(r, np.full(n, 0.7), np.zeros(n), layer))


def test_one_row_grid_and_narrow_phi(binding):
    g = eg.Geometry()
    bn = eg.Binning(n_qpt=1, qpt_min=-0.3, qpt_max=0.1, n_phi=64, threshold=2)
    check_event(binding, g, bn, eg.WORKLOADS["single_50trk"].event(3))


def test_odd_sizes_and_few_layers(binding):
    """3 layers, 77 rows, 192 columns: ragged slabs and a non-power-of-two phi axis."""
    g = eg.Geometry(radii_cm=(5.0, 30.0, 90.0), b_tesla=2.0)
    bn = eg.Binning(n_qpt=77, qpt_min=-1.3, qpt_max=0.9, n_phi=192, threshold=2, n_cot=17, n_z0=23,
                    cot_min=-3.0, cot_max=2.0, z0_min=-20.0, z0_max=10.0)
    ev = eg.simulate_event(g, 40, (0.7, 20.0), 30, seed=99)
    check_event(binding, g, bn, ev, tiling=(5, 64, 128, 1, 3))
    check_event(binding, g, bn, ev, tiling=(5, 64, 128, 0, 7))
    check_event(binding, g, bn, ev)


@pytest.mark.parametrize("n_cot,n_z0,dense", [(128, 128, True), (256, 64, False), (64, 256, False)])
def test_largest_stage2_grids(binding, n_cot, n_z0, dense):
    """Stage-2 grids of the largest size accepted (16,384 cells: 32 KB of masks for each
    confirming warp, so fewer warps share a CTA), on the pileup event cut to 30,000 hits (many
    candidates per CTA) and on a 50-track event."""
    w = eg.WORKLOADS["pileup_100k" if dense else "single_50trk"]
    ev = w.event(1).subset(np.arange(30000)) if dense else w.event(1)
    bn = eg.with_binning(w, n_cot=n_cot, n_z0=n_z0).binning
    r = check_event(binding, w.geometry, bn, ev)
    assert r["stage2_checked"] > (200 if dense else 20)
    # the same event in a batch (where a detector of ten layers takes the packed 10-bit grids)
    other = w.event(2).subset(np.arange(min(w.event(2).n_hits, 20000)))
    events = [other, ev]
    with binding.HoughBatch(w.geometry, bn, max_events=2, max_hits=other.n_hits + ev.n_hits) as b:
        b.run_events(events)
        cands, offs = b.candidates()
    assert np.array_equal(cands[offs[1]:offs[2]], r["got"]["candidates"])
    assert np.array_equal(cands[offs[0]:offs[1]], run_gpu(binding, w.geometry, bn, other)["candidates"])


def test_candidate_capacity_truncates_in_raster_order(binding):
    w = eg.WORKLOADS["single_50trk"]
    ev = w.event(0)
    ref = oracle.run(w.geometry, w.binning, ev)
    n = len(ref["candidates"])
    assert n > 10
    with binding.HoughContext(w.geometry, w.binning, max_hits=ev.n_hits, max_candidates=10) as ctx:
        ctx.vote_event(ev)
        ctx.peaks()
        ctx.stage2()
        with pytest.raises(binding.HoughError) as e:
            ctx.candidates(cap=10)
        assert e.value.code == binding.ETRUNC
        st = ctx.stats(allow_device_error=True)
        assert st.device_error & 4 and st.n_candidates == n
        out = np.zeros(10, dtype=binding.CANDIDATE_DTYPE)
        import ctypes
        nn = ctypes.c_int32(0)
        rc = binding.load().hough_get_candidates(ctx._h, out.ctypes.data, 10, ctypes.byref(nn), binding.HOST, None)
        assert rc == binding.ETRUNC and nn.value == n
        assert [(int(c["iq"]), int(c["jphi"])) for c in out] == \
            [(int(c["iq"]), int(c["jphi"])) for c in ref["candidates"][:10]]


@pytest.mark.parametrize("name, max_members", [("pileup_100k", 5000), ("paper_5000", 20000)])
def test_member_pool_overflow(binding, name, max_members):
    """A member pool smaller than the event's members (a candidate of four warps on the pileup
    event; a warp per candidate, lists in chunks, on the paper's 5,000-track event): stage 2 is
    unchanged, the pool is filled exactly, every candidate's list is either whole or flagged
    (flags bit 1) and a subset of the whole one, and the event reports HOUGH_DEVERR_MEMBERS."""
    w = eg.paper_workload(5000) if name == "paper_5000" else eg.WORKLOADS[name]
    ev = w.event(0)

    def run(mm):
        with binding.HoughContext(w.geometry, w.binning, max_hits=ev.n_hits, max_candidates=1 << 18,
                                  max_members=mm) as ctx:
            ctx.vote_event(ev)
            ctx.peaks()
            ctx.stage2()
            cands = ctx.candidates()
            off, mem = ctx.members(len(cands), allow_truncated=True)
            err = ctx.stats(allow_device_error=True).device_error
        return cands, off, mem, err

    cb, ob, mb, eb = run(1 << 22)
    cs, os_, ms, es = run(max_members)
    assert eb == 0 and es == 8   # HOUGH_DEVERR_MEMBERS: the lists were cut
    assert int(ob[-1]) == int(cb["n_members"].sum()) > max_members
    for f in ("iq", "jphi", "mask", "n_members", "icot", "jz0", "mask2"):
        assert np.array_equal(cs[f], cb[f]), f
    assert np.array_equal(cs["flags"] & 1, cb["flags"] & 1) and not (cb["flags"] & 2).any()
    counts = np.diff(os_)
    assert int(counts.sum()) == max_members
    cut = (cs["flags"] & 2) != 0
    assert cut.any() and np.array_equal(cut, counts < cs["n_members"])
    for q in range(len(cs)):
        got, full = ms[os_[q]:os_[q + 1]], mb[ob[q]:ob[q + 1]]
        if cut[q]:
            assert np.isin(got, full).all()
        else:
            assert np.array_equal(got, full)


def test_bad_hits(binding):
    """Host buffers: a bad hit is rejected with HOUGH_EINVAL before any work.  Device buffers: it
    is dropped on the device, flagged in device_error, and the other hits vote as usual."""
    w = eg.WORKLOADS["single_50trk"]
    ev = w.event(1)
    bad = _event(np.r_[ev.r, 30.0, -1.0], np.r_[ev.phi, 0.1, 0.2], np.r_[ev.z, 0, 0], np.r_[ev.layer, 12, 3])
    with binding.HoughContext(w.geometry, w.binning, max_hits=bad.n_hits) as ctx:
        with pytest.raises(binding.HoughError) as e:
            ctx.vote_event(bad)
        assert e.value.code == binding.EINVAL
        import torch
        t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (bad.r, bad.phi, bad.z, bad.layer)]
        ctx.vote(*t, n_hits=bad.n_hits, where=binding.DEVICE)
        ctx.peaks()
        st = ctx.stats(allow_device_error=True)
        assert st.device_error == 1 | 2 and st.n_hits == ev.n_hits
        M = ctx.accumulator()
    ref = oracle.run(w.geometry, w.binning, ev)
    assert_accumulator_parity(M, ref["M"], ref["vote_flags"])


def test_capacity_error(binding):
    w = eg.WORKLOADS["single_50trk"]
    ev = w.event(0)
    with binding.HoughContext(w.geometry, w.binning, max_hits=ev.n_hits - 1) as ctx:
        with pytest.raises(binding.HoughError) as e:
            ctx.vote_event(ev)
        assert e.value.code == binding.ECAPACITY


def test_process_from_host_memory(binding):
    """hough_process on host hits (checked on the device, candidates through mapped memory): the
    same candidates as the step-by-step calls, repeatable, a truncated copy on a small capacity,
    and HOUGH_EINVAL for an event with a bad hit."""
    w = eg.WORKLOADS["pileup_100k"]
    ev = w.event(4)
    ref = run_gpu(binding, w.geometry, w.binning, ev)["candidates"]
    with binding.HoughContext(w.geometry, w.binning, max_hits=ev.n_hits, max_candidates=1 << 16) as ctx:
        for _ in range(2):
            got = ctx.process(ev.r, ev.phi, ev.z, ev.layer)
            assert np.array_equal(got, ref)
        out = np.zeros(len(ref), dtype=binding.CANDIDATE_DTYPE)
        with pytest.raises(binding.HoughError) as e:
            ctx.process(ev.r, ev.phi, ev.z, ev.layer, cap=10, out=out)
        assert e.value.code == binding.ETRUNC
        assert np.array_equal(out[:10], ref[:10])
        bad = ev.subset(np.arange(ev.n_hits))
        bad.z[777] = np.float32(np.inf)
        with pytest.raises(binding.HoughError) as e:
            ctx.process(bad.r, bad.phi, bad.z, bad.layer)
        assert e.value.code == binding.EINVAL
        assert np.array_equal(ctx.process(ev.r, ev.phi, ev.z, ev.layer), ref)


def test_process_reads_pinned_hits_in_place(binding):
    """Pinned host hits are read by the staging kernels in place (no copy); the result equals the
    pageable-memory path (copied), also through hough_vote with its host check, and a bad pinned
    hit is still rejected."""
    torch = pytest.importorskip("torch")
    w = eg.WORKLOADS["pileup_100k"]
    ev = w.event(6)
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (ev.r, ev.phi, ev.z, ev.layer)]
    with binding.HoughContext(w.geometry, w.binning, max_hits=ev.n_hits, max_candidates=1 << 16) as ctx:
        ref = ctx.process(ev.r, ev.phi, ev.z, ev.layer).copy()
        got = ctx.process(*pinned, n_hits=ev.n_hits)
        assert np.array_equal(got, ref)
        M_ref = ctx.accumulator()
        ctx.vote(*pinned, n_hits=ev.n_hits, where=binding.HOST)
        ctx.peaks()
        ctx.stage2()
        assert np.array_equal(ctx.accumulator(), M_ref)
        assert np.array_equal(ctx.candidates(), ref)
        pinned[0][123] = -1.0
        with pytest.raises(binding.HoughError) as e:
            ctx.process(*pinned, n_hits=ev.n_hits)
        assert e.value.code == binding.EINVAL
        with pytest.raises(binding.HoughError) as e:
            ctx.vote(*pinned, n_hits=ev.n_hits, where=binding.HOST)
        assert e.value.code == binding.EINVAL


def test_back_to_back_events_on_one_context(binding):
    """Events put through one context with nothing between one event's stage 2 and the next
    event's vote (the next event's counting then runs beside the last confirmation): the last
    event's results equal those of a context that saw it alone."""
    import torch
    w = eg.WORKLOADS["pileup_100k"]
    evs = [w.event(7), w.event(8).subset(np.arange(20000)), w.event(9)]
    dev = [[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (e.r, e.phi, e.z, e.layer)] for e in evs]
    torch.cuda.synchronize()
    n_max = max(e.n_hits for e in evs)
    with binding.HoughContext(w.geometry, w.binning, max_hits=n_max) as ctx:
        for k, e in enumerate(evs):
            ctx.vote(*dev[k], n_hits=e.n_hits, where=binding.DEVICE)
            ctx.peaks()
            ctx.stage2()
        cands = ctx.candidates()
        st = ctx.stats()
        off, mem = ctx.members(len(cands))
        M = ctx.accumulator()
    alone = run_gpu(binding, w.geometry, w.binning, evs[-1], where="device")
    assert np.array_equal(M, alone["M"])
    assert np.array_equal(cands, alone["candidates"])
    assert np.array_equal(off, alone["member_offsets"]) and np.array_equal(mem, alone["members"])
    for f in ("votes", "n_candidates", "n_members", "stage2_votes"):
        assert int(getattr(st, f)) == int(getattr(alone["stats"], f)), f
