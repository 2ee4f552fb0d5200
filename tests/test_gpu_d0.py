"""The impact-parameter axis d0 on the GPU (needs a GPU): non-prompt tracks, a (d0, q/pT, phi0)
grid stored as n_d0 slices of stacked rows, the 3 x 3 x 3 peak rule.

Every cell is compared with the FP64 oracle (equal up to the votes it flags), then the candidate
list, member lists and stage-2 results; plus the per-vote FP64 path of layers at several radii,
every vote and peak configuration, the count accumulator, batches and the allocation-free vote."""
import numpy as np
import pytest

import oracle
from paper_1310_7556_gb300 import eventgen as eg

from parity import assert_accumulator_parity, assert_candidate_parity, stacked
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


def _small_d0(**kw):
    """The 50-track workload on a 5 x 128 x 256 grid, d0 bins over [-1, 1] cm."""
    w = eg.WORKLOADS["single_50trk"]
    return eg.with_binning(w, **{"n_d0": 5, "d0_min": -1.0, "d0_max": 1.0, **kw})


@pytest.mark.parametrize("index", range(2))
def test_displaced_event_full_size(binding, index):
    """200 displaced tracks (d0 ~ U(-2, 2) cm) + 1,000 noise hits on the 16 x 256 x 2048 grid."""
    w = eg.WORKLOADS["displaced_d0"]
    r = check_event(binding, w.geometry, w.binning, w.event(index))
    cands = r["got"]["candidates"]
    assert len(cands) > 100 and len(np.unique(cands["iq"] // w.binning.n_qpt)) > w.binning.n_d0 // 2
    assert r["stage2_checked"] > 50


@pytest.mark.parametrize("index", range(2))
def test_prompt_event_on_a_d0_grid(binding, index):
    w = _small_d0()
    r = check_event(binding, w.geometry, w.binning, w.event(index))
    assert r["stage2_checked"] > 0


def test_d0_counts(binding):
    """The count accumulator on the displaced workload's grid."""
    w = eg.with_binning(eg.WORKLOADS["displaced_d0"], accumulator=eg.ACC_COUNTS, threshold=8)
    r = check_event(binding, w.geometry, w.binning, w.event(2))
    assert len(r["got"]["candidates"]) > 100


def test_d0_per_vote_path(binding):
    """Layers whose hits lie at several radii: every vote of theirs is decided in FP64 on a d0 grid."""
    w = eg.WORKLOADS["displaced_d0"]
    ev = w.event(3).subset(np.arange(3000))
    rng = np.random.default_rng(8)
    jitter = ev.layer % 3 == 0
    ev.r = np.where(jitter, ev.r + rng.uniform(-0.3, 0.3, ev.n_hits), ev.r).astype(np.float32)
    r = check_event(binding, w.geometry, w.binning, ev)
    st = r["got"]["stats"]
    assert st.uniform_layers != (1 << 10) - 1 and st.general_votes > 0


def test_centred_slice_equals_the_prompt_grid(binding):
    """n_d0 = 3 over [-1.5, 1.5] cm: the middle slice has d0 = 0 exactly and equals the prompt grid."""
    w = eg.WORKLOADS["pileup_100k"]
    ev = w.event(1).subset(np.arange(30000))
    prompt = run_gpu(binding, w.geometry, w.binning, ev)
    w3 = eg.with_binning(w, n_d0=3, d0_min=-1.5, d0_max=1.5)
    three = run_gpu(binding, w3.geometry, w3.binning, ev)
    q = w.binning.n_qpt
    assert np.array_equal(three["M"][q:2 * q], prompt["M"])


@pytest.mark.parametrize("tiling", [dict(vote_mode=1), dict(vote_mode=1, tile_qpt=7, tile_phi=128, threads=512),
                                    dict(vote_mode=1, tile_qpt=32, tile_phi=2048, threads=1024),
                                    dict(gather_rows=16, gather_cols=256, gather_threads=512),
                                    dict(gather_rows=3, gather_cols=1024, gather_threads=1024),
                                    dict(band_rows=1), dict(band_rows=3), dict(band_rows=7), dict(band_rows=16)])
def test_d0_configurations_agree_bit_for_bit(binding, tiling):
    """Gather and scatter votes, tiles straddling d0 slices (ragged by 7 and 3 rows), and peak bands
    of 1 to 16 rows (ragged at each slice's end by 3 and 7), one result."""
    w = eg.WORKLOADS["displaced_d0"]
    ev = w.event(1)
    base = run_gpu(binding, w.geometry, w.binning, ev)
    other = run_gpu(binding, w.geometry, w.binning, ev, tiling=tiling)
    assert np.array_equal(base["M"], other["M"])
    assert np.array_equal(base["candidates"], other["candidates"])


def test_d0_grid_too_wide_is_refused(binding):
    """Nine rows of 32768 counts do not fit in shared memory: the axes are refused at creation."""
    w = eg.with_binning(_small_d0(), n_phi=32768, accumulator=eg.ACC_COUNTS)
    with pytest.raises(binding.HoughError) as e:
        binding.HoughContext(w.geometry, w.binning, max_hits=16)
    assert e.value.code == binding.EINVAL


def test_d0_batch_equals_events_alone(binding):
    w = eg.WORKLOADS["displaced_d0"]
    empty = eg.Event(np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(0, np.float32),
                     np.zeros(0, np.uint8), np.zeros(0, np.int32))
    events = [w.event(0), empty, w.event(1).subset(np.arange(1500)), w.event(2)]
    total = sum(e.n_hits for e in events)
    with binding.HoughBatch(w.geometry, w.binning, max_events=len(events), max_hits=total) as b:
        b.run_events(events)
        cands, offs = b.candidates()
        for e, ev in enumerate(events):
            alone = run_gpu(binding, w.geometry, w.binning, ev, max_candidates=1 << 17)
            assert np.array_equal(b.accumulator(e), alone["M"]), f"event {e}"
            assert np.array_equal(cands[offs[e]:offs[e + 1]], alone["candidates"]), f"event {e}"
        ref = oracle.run(w.geometry, w.binning, events[3])
        assert_accumulator_parity(b.accumulator(3), ref["M"], ref["vote_flags"])
        assert_candidate_parity(cands[offs[3]:offs[4]], stacked(ref["candidates"], w.binning.n_qpt),
                                ref["vote_flags"], w.binning.n_phi, q_rows=w.binning.n_qpt)


def test_d0_static_vote(binding):
    torch = pytest.importorskip("torch")
    w = _small_d0()
    ev = w.event(5)
    dev = torch.device("cuda", 0)
    hits = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (ev.r, ev.phi, ev.z, ev.layer)]
    acc = torch.full((binding.grid_rows(w.binning), w.binning.n_phi), -1, dtype=torch.int16, device=dev)
    binding.vote_static(w.geometry, w.binning, *hits, ev.n_hits, acc, stream=torch.cuda.current_stream(dev))
    torch.cuda.synchronize()
    got = acc.cpu().numpy().view(np.uint16)
    assert np.array_equal(got, run_gpu(binding, w.geometry, w.binning, ev)["M"])


def test_single_d0_slice_at_zero_is_the_prompt_path(binding):
    """One d0 bin centred on 0 (d0 = 0 exactly): the accumulator, the 3x3x3 peak rule with no
    neighbouring slices and stage 2 reduce to the prompt path's, result for result."""
    w = eg.WORKLOADS["pileup_100k"]
    ev = w.event(2).subset(np.arange(30000))
    prompt = run_gpu(binding, w.geometry, w.binning, ev)
    w1 = eg.with_binning(w, n_d0=1, d0_min=-0.5, d0_max=0.5)
    one = run_gpu(binding, w1.geometry, w1.binning, ev)
    assert np.array_equal(one["M"], prompt["M"])
    assert np.array_equal(one["candidates"], prompt["candidates"])


def test_d0_odd_sizes_and_few_layers(binding):
    """3 layers at 5, 30 and 90 cm, 3 d0 bins over +-4 cm, 77 x 192 cells per slice, odd stage-2
    axes; displaced tracks (d0 within +-3 cm), with the default, a gather and a scatter tiling."""
    g = eg.Geometry(radii_cm=(5.0, 30.0, 90.0), b_tesla=2.0)
    bn = eg.Binning(n_qpt=77, qpt_min=-1.3, qpt_max=0.9, n_phi=192, threshold=2, n_cot=17, n_z0=23,
                    cot_min=-3.0, cot_max=2.0, z0_min=-20.0, z0_max=10.0, n_d0=3, d0_min=-4.0, d0_max=4.0)
    ev = eg.simulate_event(g, 40, (0.7, 20.0), 30, seed=98, d0_range=(-3.0, 3.0))
    for t in (None, dict(gather_rows=5, gather_cols=64, band_rows=3), dict(vote_mode=1, tile_qpt=5, tile_phi=64)):
        check_event(binding, g, bn, ev, tiling=t)
