"""The error path of the device-side bounded wait, made to run without faulting the GPU (needs a GPU).

The gather vote's CTAs copy slices of the bucket profile into shared memory with bulk copies and
wait for them on an mbarrier with a bound of about a second.  hough_set_copy_wait(ctx, -1) makes the
first bound of every such wait expire at once: each CTA then sets HOUGH_DEVERR_TIMEOUT, waits once
more with the full bound for its own copies to land, and writes nothing.  The test checks that the
expiry is reported (hough_get_stats returns HOUGH_EDEVICE with the bit set) and that the context
keeps working afterwards.
"""
import numpy as np
import pytest

from paper_1310_7556_gb300 import eventgen as eg

pytestmark = pytest.mark.gpu

DEVERR_TIMEOUT = 16


@pytest.fixture(scope="module")
def binding():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1310_7556_gb300 import binding as b
    b.load()
    return b


@pytest.mark.parametrize("mode", ["gather", "fused"])
def test_expired_copy_wait_is_reported_and_the_context_stays_usable(binding, mode):
    w = eg.WORKLOADS["pileup_100k"]
    ev = w.event(0)
    with binding.HoughContext(w.geometry, w.binning, max_hits=ev.n_hits) as ctx:
        if mode == "fused":
            ctx.set_tiling(vote_mode=binding.VOTE_FUSED, band_rows=4)
        ctx.vote_event(ev)
        ctx.peaks()
        ref = ctx.candidates().copy()
        assert ctx.stats().device_error == 0
        ctx.set_copy_wait(-1)
        ctx.vote_event(ev)
        ctx.peaks()
        with pytest.raises(binding.HoughError) as e:
            ctx.stats()
        assert e.value.code == binding.EDEVICE
        assert ctx.stats(allow_device_error=True).device_error == DEVERR_TIMEOUT
        ctx.set_copy_wait(0)
        ctx.vote_event(ev)
        ctx.peaks()
        assert ctx.stats().device_error == 0
        assert np.array_equal(ctx.candidates(), ref)
