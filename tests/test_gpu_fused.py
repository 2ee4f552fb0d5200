"""The fused vote and peak search (vote_mode HOUGH_VOTE_FUSED; needs a GPU): a CTA per band of
full rows computes the band's cells and its two halo rows in shared memory and searches them for
peaks there, so the accumulator never goes to device memory.  Its candidates, member lists and
stage-2 results must equal the default path's bit for bit (and the oracle's up to flagged votes)
for every band height and block size, with the fallback of layers whose hits lie at several
radii, in batches and through hough_process."""
import numpy as np
import pytest

import oracle
from paper_1310_7556_gb300 import eventgen as eg

from parity import assert_candidate_parity, assert_members_and_stage2_parity, stacked
from test_gpu_parity import run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1310_7556_gb300 import binding as b
    b.load()
    return b


def run_fused(binding, geometry, binning, ev, band_rows=4, threads=256):
    with binding.HoughContext(geometry, binning, max_hits=max(ev.n_hits, 1), max_candidates=1 << 18) as ctx:
        ctx.set_tiling(vote_mode=binding.VOTE_FUSED, band_rows=band_rows, gather_threads=threads)
        ctx.vote_event(ev)
        ctx.peaks()
        ctx.stage2()
        cands = ctx.candidates()
        st = ctx.stats()
        off, mem = ctx.members(len(cands))
        with pytest.raises(binding.HoughError) as e:
            ctx.accumulator()
        assert e.value.code == binding.ENOTREADY
    return dict(candidates=cands, stats=st, member_offsets=off, members=mem)


def _same(a, b):
    assert np.array_equal(a["candidates"], b["candidates"])
    assert np.array_equal(a["member_offsets"], b["member_offsets"]) and np.array_equal(a["members"], b["members"])
    assert int(a["stats"].votes) == int(b["stats"].votes)


@pytest.mark.parametrize("band_rows,threads", [(1, 256), (3, 512), (4, 256), (7, 1024), (16, 256)])
def test_pileup_event_equals_the_default_path(binding, band_rows, threads):
    """The 100k-hit pileup event (512 x 2048): band heights 1 to 16 (ragged last bands for 3 and
    7), 256 to 1024 threads."""
    w = eg.WORKLOADS["pileup_100k"]
    ev = w.event(0)
    _same(run_fused(binding, w.geometry, w.binning, ev, band_rows, threads), run_gpu(binding, w.geometry, w.binning, ev))


@pytest.mark.parametrize("name,index", [("single_50trk", 2), ("pileup_100k", 3)])
def test_fused_against_the_oracle(binding, name, index):
    w = eg.WORKLOADS[name]
    ev = w.event(index)
    ref = oracle.run(w.geometry, w.binning, ev)
    got = run_fused(binding, w.geometry, w.binning, ev)
    assert_candidate_parity(got["candidates"], stacked(ref["candidates"], w.binning.n_qpt), ref["vote_flags"],
                            w.binning.n_phi)
    assert assert_members_and_stage2_parity(got["candidates"], got["member_offsets"], got["members"], ref,
                                            w.binning.threshold, w.geometry.n_layers) > 0


def test_paper_grid_and_odd_sizes(binding):
    """The paper's 2048 x 2048 grid (5,000 helices), and 3 layers on 77 x 192 cells (a phi axis
    that is not a multiple of 256 and a ragged last band)."""
    w = eg.paper_workload(5000)
    ev = w.event(0)
    _same(run_fused(binding, w.geometry, w.binning, ev, 8), run_gpu(binding, w.geometry, w.binning, ev))
    g = eg.Geometry(radii_cm=(5.0, 30.0, 90.0), b_tesla=2.0)
    bn = eg.Binning(n_qpt=77, qpt_min=-1.3, qpt_max=0.9, n_phi=192, threshold=2, n_cot=17, n_z0=23,
                    cot_min=-3.0, cot_max=2.0, z0_min=-20.0, z0_max=10.0)
    ev = eg.simulate_event(g, 40, (0.7, 20.0), 30, seed=99)
    for r in (1, 4, 5):
        _same(run_fused(binding, g, bn, ev, r), run_gpu(binding, g, bn, ev))


def test_layers_of_several_radii_fall_back_to_the_peak_kernel(binding):
    """Jittered radii on three layers: their votes come from the scatter kernel after the fused
    kernel, which then hands its rows to the peak kernel; the result is the default path's."""
    w = eg.WORKLOADS["pileup_100k"]
    ev = w.event(4).subset(np.arange(40000))
    rng = np.random.default_rng(21)
    jitter = ev.layer % 3 == 1
    ev.r = np.where(jitter, ev.r + rng.uniform(-0.3, 0.3, ev.n_hits), ev.r).astype(np.float32)
    got = run_fused(binding, w.geometry, w.binning, ev)
    assert got["stats"].uniform_layers != (1 << 10) - 1
    _same(got, run_gpu(binding, w.geometry, w.binning, ev))


def test_batch_and_process(binding):
    """A batch of eight events of the batch workload under the fused mode equals the default
    batch, and hough_process under the fused mode equals the default one."""
    w = eg.WORKLOADS["batch_256"]
    events = [w.event(i) for i in range(8)]
    total = sum(e.n_hits for e in events)
    out = {}
    for mode in (binding.VOTE_GATHER, binding.VOTE_FUSED):
        with binding.HoughBatch(w.geometry, w.binning, max_events=len(events), max_hits=total) as b:
            b.set_tiling(vote_mode=mode, band_rows=8)
            b.run_events(events)
            out[mode] = b.candidates()
            if mode == binding.VOTE_FUSED:
                with pytest.raises(binding.HoughError) as e:
                    b.accumulator(0)
                assert e.value.code == binding.ENOTREADY
    assert np.array_equal(out[binding.VOTE_GATHER][0], out[binding.VOTE_FUSED][0])
    assert np.array_equal(out[binding.VOTE_GATHER][1], out[binding.VOTE_FUSED][1])
    wp = eg.WORKLOADS["pileup_100k"]
    ev = wp.event(5)
    res = {}
    for mode in (binding.VOTE_GATHER, binding.VOTE_FUSED):
        with binding.HoughContext(wp.geometry, wp.binning, max_hits=ev.n_hits, max_candidates=1 << 18) as ctx:
            ctx.set_tiling(vote_mode=mode, band_rows=4)
            res[mode] = ctx.process(ev.r, ev.phi, ev.z, ev.layer, ev.n_hits).copy()
    assert len(res[binding.VOTE_FUSED]) > 100
    assert np.array_equal(res[binding.VOTE_GATHER], res[binding.VOTE_FUSED])


def test_fused_mode_is_refused_where_it_does_not_apply(binding):
    """The count accumulator and a d0 axis keep the separate peak search."""
    w = eg.WORKLOADS["single_50trk"]
    for bn in (eg.with_binning(w, accumulator=eg.ACC_COUNTS).binning,
               eg.with_binning(w, n_d0=3, d0_min=-1.0, d0_max=1.0).binning):
        with binding.HoughContext(w.geometry, bn, max_hits=64) as ctx:
            with pytest.raises(binding.HoughError) as e:
                ctx.set_tiling(vote_mode=binding.VOTE_FUSED)
            assert e.value.code == binding.EINVAL
