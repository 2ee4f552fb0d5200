"""The count accumulator on the GPU (needs a GPU): a cell holds its number of votes, the literal
A[B[i]] += 1 of Sec. 8, saturating at 65535, and the peak search reads the count.  It is voted by
a gather (per cell, the hits of two buckets compared with the row's table fraction; the default)
or by the paper's shared-memory atomic scatter, bit for bit alike.

Every count is compared with the FP64 oracle cell by cell (equal up to the votes the oracle flags
as within its edge window), then the candidates, member lists and stage-2 results as for the
layer accumulator; plus the properties that tie the two accumulators together, saturation, every
scatter tile shape, the batched path and the allocation-free entry point."""
import numpy as np
import pytest

import oracle
from paper_1310_7556_gb300 import eventgen as eg

from parity import assert_count_parity, assert_candidate_parity
from test_gpu_parity import check_event, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1310_7556_gb300 import binding as b
    b.load()
    return b


def _counts(w, threshold):
    return eg.with_binning(w, accumulator=eg.ACC_COUNTS, threshold=threshold)


def _popcount(a):
    a = np.asarray(a, dtype=np.uint16)
    return np.unpackbits(a.view(np.uint8)).reshape(a.shape + (16,)).sum(-1)


@pytest.mark.parametrize("index", range(3))
def test_single_event_counts(binding, index):
    w = _counts(eg.WORKLOADS["single_50trk"], 8)
    r = check_event(binding, w.geometry, w.binning, w.event(index))
    assert r["stage2_checked"] > 0


def test_pileup_event_counts_full_size(binding):
    """The 100k-hit pileup event on its 512 x 2048 grid: about 48 votes per cell, so the count
    threshold sits near the top of the noise (70) and thousands of cells pass it."""
    w = _counts(eg.WORKLOADS["pileup_100k"], 70)
    r = check_event(binding, w.geometry, w.binning, w.event(0))
    assert len(r["got"]["candidates"]) > 1000 and r["stage2_checked"] > 500


@pytest.mark.parametrize("n_tracks", [100, 1000])
def test_paper_grid_counts(binding, n_tracks):
    """The paper's detector and 2048 x 2048 grid with a count threshold of 8 hits."""
    w = _counts(eg.paper_workload(n_tracks), 8)
    check_event(binding, w.geometry, w.binning, w.event(0))


def test_per_vote_path_counts(binding):
    """Hits of a layer at different radii take the FP32 asinf path with FP64 edge refinement."""
    w = _counts(eg.WORKLOADS["pileup_100k"], 30)
    ev = w.event(3).subset(np.arange(20000))
    rng = np.random.default_rng(5)
    ev.r = (ev.r + rng.uniform(-0.5, 0.5, ev.n_hits)).astype(np.float32)
    r = check_event(binding, w.geometry, w.binning, ev)
    st = r["got"]["stats"]
    assert st.uniform_layers == 0 and st.refined_votes > 0


def test_counts_and_layer_masks_agree_on_occupancy(binding):
    """The same event through both accumulators: a cell is occupied in one exactly when in the
    other, its count is at least its number of layers, and the counts sum to the votes cast."""
    w = eg.WORKLOADS["pileup_100k"]
    ev = w.event(1).subset(np.arange(30000))
    layers = run_gpu(binding, w.geometry, w.binning, ev)
    wc = _counts(w, 40)
    counts = run_gpu(binding, wc.geometry, wc.binning, ev)
    Ml, Mc = layers["M"], counts["M"]
    assert np.array_equal(Mc > 0, Ml != 0)
    assert np.all(Mc >= _popcount(Ml))
    assert int(Mc.astype(np.int64).sum()) == int(counts["stats"].votes) == int(layers["stats"].votes)


def test_counts_saturate_at_65535(binding):
    """70,000 copies of one hit: each cell it votes in holds 65535, as in the oracle."""
    n = 70000
    ev = eg.Event(np.full(n, 30.0, np.float32), np.full(n, 0.3, np.float32), np.zeros(n, np.float32),
                  np.zeros(n, np.uint8), np.zeros(n, np.int32))
    bn = eg.Binning(n_qpt=2, qpt_min=-0.5, qpt_max=0.5, n_phi=64, threshold=1, accumulator=eg.ACC_COUNTS)
    got = run_gpu(binding, eg.Geometry(), bn, ev)
    ref, _, flags = oracle.vote(oracle.make_binning(eg.Geometry(), bn), ev)
    assert len(flags) == 0
    assert np.array_equal(got["M"], ref) and sorted(got["M"][got["M"] > 0].tolist()) == [65535, 65535]
    assert int(got["stats"].votes) == 2 * n


@pytest.mark.parametrize("tiling", [dict(vote_mode=1, tile_qpt=1, tile_phi=64, threads=128),
                                    dict(vote_mode=1, tile_qpt=7, tile_phi=128),
                                    dict(vote_mode=1, tile_qpt=16, tile_phi=256, threads=512),
                                    dict(vote_mode=1, tile_qpt=32, tile_phi=512, threads=1024),
                                    dict(vote_mode=1, tile_qpt=3, tile_phi=2048, threads=256),
                                    dict(gather_rows=1, gather_cols=64, gather_threads=256),
                                    dict(gather_rows=7, gather_cols=256, gather_threads=512),
                                    dict(gather_rows=32, gather_cols=1024, gather_threads=1024),
                                    dict(gather_rows=3, gather_cols=2048, gather_threads=256),
                                    dict(band_rows=5), dict(band_rows=16)])
def test_count_tilings_agree_bit_for_bit(binding, tiling):
    """Every scatter tile (ragged last slabs of 512 rows by 7 and 3 rows), every count-gather tile
    (ragged row bands; windows staged, too full for their slot, and wider than the ring, both read
    from global memory) and band height gives the same counts and candidates."""
    w = _counts(eg.WORKLOADS["pileup_100k"], 40)
    ev = w.event(2).subset(np.arange(40000))
    base = run_gpu(binding, w.geometry, w.binning, ev)
    other = run_gpu(binding, w.geometry, w.binning, ev, tiling=tiling)
    assert np.array_equal(base["M"], other["M"])
    assert np.array_equal(base["candidates"], other["candidates"])


def test_count_gather_is_the_default(binding):
    w = _counts(eg.WORKLOADS["single_50trk"], 8)
    with binding.HoughContext(w.geometry, w.binning, max_hits=16) as ctx:
        assert ctx.get_tiling()["vote_mode"] == binding.VOTE_GATHER


@pytest.mark.parametrize("vote_mode", [0, 1])
def test_counts_mixed_uniform_and_non_uniform_layers(binding, vote_mode):
    """Layers of one radius counted by the gather (or the scatter), the others added by the scatter."""
    w = _counts(eg.WORKLOADS["pileup_100k"], 40)
    ev = w.event(7).subset(np.arange(25000))
    jitter = ev.layer % 2 == 1
    ev.r = np.where(jitter, ev.r * np.float32(1.003), ev.r).astype(np.float32)
    ev.r[np.nonzero(jitter)[0][::2]] *= np.float32(0.999)
    r = check_event(binding, w.geometry, w.binning, ev, tiling=dict(vote_mode=vote_mode))
    assert r["got"]["stats"].uniform_layers == 0b0101010101


def test_count_threshold_range(binding):
    """A count threshold may exceed the 16 layers the layer accumulator allows."""
    w = _counts(eg.WORKLOADS["pileup_100k"], 75)
    ev = w.event(0)
    ref = oracle.run(w.geometry, w.binning, ev)
    got = run_gpu(binding, w.geometry, w.binning, ev)
    assert_candidate_parity(got["candidates"], ref["candidates"], ref["vote_flags"], w.binning.n_phi)
    assert len(got["candidates"]) > 0 and int(got["candidates"]["mask"].min()) >= 75
    bad = eg.with_binning(eg.WORKLOADS["single_50trk"], threshold=17)
    with pytest.raises(binding.HoughError):
        binding.HoughContext(bad.geometry, bad.binning, max_hits=16)


def test_batch_counts_equal_events_alone(binding):
    """Uneven events (4k to 24k hits, one of 7 hits, one empty; none to 13k candidates) in one
    batch: each equals the single-event path, and the largest matches the oracle."""
    w = _counts(eg.WORKLOADS["batch_256"], 20)
    empty = eg.Event(np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(0, np.float32),
                     np.zeros(0, np.uint8), np.zeros(0, np.int32))
    events = [w.event(1), w.event(2), empty, w.event(3), w.event(2).subset(np.arange(7))]
    total = sum(e.n_hits for e in events)
    with binding.HoughBatch(w.geometry, w.binning, max_events=len(events), max_hits=total) as b:
        b.run_events(events)
        cands, offs = b.candidates()
        for e, ev in enumerate(events):
            alone = run_gpu(binding, w.geometry, w.binning, ev, max_candidates=1 << 17)
            assert np.array_equal(b.accumulator(e), alone["M"]), f"event {e}"
            assert np.array_equal(cands[offs[e]:offs[e + 1]], alone["candidates"]), f"event {e}"
        ref = oracle.run(w.geometry, w.binning, events[3])
        assert_count_parity(b.accumulator(3), ref["M"], ref["vote_flags"])
        assert_candidate_parity(cands[offs[3]:offs[4]], ref["candidates"], ref["vote_flags"], w.binning.n_phi)
        assert offs[4] - offs[3] > 10000


def test_static_vote_counts(binding):
    torch = pytest.importorskip("torch")
    w = _counts(eg.WORKLOADS["pileup_100k"], 40)
    ev = w.event(4).subset(np.arange(50000))
    dev = torch.device("cuda", 0)
    hits = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (ev.r, ev.phi, ev.z, ev.layer)]
    acc = torch.full((w.binning.n_qpt, w.binning.n_phi), -1, dtype=torch.int16, device=dev)
    binding.vote_static(w.geometry, w.binning, *hits, ev.n_hits, acc, stream=torch.cuda.current_stream(dev))
    torch.cuda.synchronize()
    got = acc.cpu().numpy().view(np.uint16)
    assert np.array_equal(got, run_gpu(binding, w.geometry, w.binning, ev)["M"])


def _ev(r, phi, z, layer):
    return eg.Event(np.asarray(r, np.float32), np.asarray(phi, np.float32), np.asarray(z, np.float32),
                    np.asarray(layer, np.uint8), np.zeros(len(r), np.int32))


def test_count_edge_cases(binding):
    """Empty event, single hits at the extreme azimuths, 20,000 hits at one azimuth (one bucket
    holds more hits than the gather's staging slot: read from global memory), a one-row grid and a
    3-layer, 77 x 192 grid with odd stage-2 axes -- counts by gather and by scatter."""
    w = _counts(eg.WORKLOADS["pileup_100k"], 3)
    got = run_gpu(binding, w.geometry, w.binning, _ev([], [], [], []))
    assert not got["M"].any() and len(got["candidates"]) == 0
    pi32 = np.float32(np.pi)
    for phi in (0.0, pi32, -pi32, np.nextafter(pi32, np.float32(0)), 999.0, -999.0):
        check_event(binding, w.geometry, w.binning, _ev([110.0], [phi], [0.0], [9]))
    n = 20000
    layer = np.arange(n) % 10
    r = np.asarray(w.geometry.radii_cm, np.float32)[layer]
    hot = _ev(r, np.full(n, 0.7), np.zeros(n), layer)
    for mode in (0, 1):
        check_event(binding, w.geometry, w.binning, hot, tiling=dict(vote_mode=mode))
    g = eg.Geometry()
    bn = eg.Binning(n_qpt=1, qpt_min=-0.3, qpt_max=0.1, n_phi=64, threshold=2, accumulator=eg.ACC_COUNTS)
    check_event(binding, g, bn, eg.WORKLOADS["single_50trk"].event(3))
    g3 = eg.Geometry(radii_cm=(5.0, 30.0, 90.0), b_tesla=2.0)
    bn3 = eg.Binning(n_qpt=77, qpt_min=-1.3, qpt_max=0.9, n_phi=192, threshold=2, n_cot=17, n_z0=23,
                     cot_min=-3.0, cot_max=2.0, z0_min=-20.0, z0_max=10.0, accumulator=eg.ACC_COUNTS)
    ev3 = eg.simulate_event(g3, 40, (0.7, 20.0), 30, seed=99)
    for t in (dict(gather_rows=5, gather_cols=64), dict(vote_mode=1, tile_qpt=5, tile_phi=64)):
        check_event(binding, g3, bn3, ev3, tiling=t)
