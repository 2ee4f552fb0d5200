"""hough_vote_static, the entry point that allocates nothing (needs a GPU).

Callers such as a trigger's real-time event loop may not allocate device memory once running
(cudaMalloc and cudaFree can stall the whole device for an unbounded time), so they cannot create
a hough_ctx.  hough_vote_static runs the same staging and vote kernels with their scratch in one
fixed device array of the library.  These tests call it through the C ABI and check its
accumulator against the context-based hough_vote + hough_get_accumulator, bit for bit (the masks
are integers), on consecutive calls that reuse the array with different events and axes; they
check that calls after the first allocate no device memory, and that a misaligned accumulator
is refused before any work.

The file name makes pytest collect it last; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_1310_7556_gb300 import eventgen as eg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1310_7556_gb300 import binding
    binding.load()
    torch.cuda.set_device(0)
    return torch, binding


def _context_accumulator(binding, w, ev):
    with binding.HoughContext(w.geometry, w.binning, max_hits=max(ev.n_hits, 1)) as ctx:
        ctx.vote_event(ev)
        return ctx.accumulator()


def _static_accumulator(torch, binding, w, ev):
    dev = torch.device("cuda", 0)
    hits = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (ev.r, ev.phi, ev.z, ev.layer)]
    # start from a full buffer, so that every cell the call does not write would show up
    acc = torch.full((w.binning.n_qpt, w.binning.n_phi), -1, dtype=torch.int16, device=dev)
    err = torch.full((1,), 12345, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    binding.vote_static(w.geometry, w.binning, *hits, ev.n_hits, acc, err, stream=stream)
    torch.cuda.synchronize()
    return acc.cpu().numpy().view(np.uint16), int(err.item())


def test_static_vote_matches_context_vote_on_consecutive_calls(env):
    torch, binding = env
    pileup = eg.WORKLOADS["pileup_100k"]
    small = eg.WORKLOADS["single_50trk"]
    calls = [(pileup, pileup.event(0)), (small, small.event(1)), (pileup, pileup.event(4)),
             (pileup, pileup.event(4))]
    for w, ev in calls:
        got, err = _static_accumulator(torch, binding, w, ev)
        assert err == 0
        assert np.array_equal(got, _context_accumulator(binding, w, ev))


def test_static_vote_non_uniform_radii_and_empty_event(env):
    torch, binding = env
    w = eg.WORKLOADS["pileup_100k"]
    ev = w.event(6).subset(np.arange(15000))
    ev.r = (ev.r + np.random.default_rng(2).uniform(-0.3, 0.3, ev.n_hits)).astype(np.float32)
    for e in (ev, ev.subset(np.arange(0))):
        got, err = _static_accumulator(torch, binding, w, e)
        assert err == 0
        assert np.array_equal(got, _context_accumulator(binding, w, e))


def test_static_vote_rejects_sizes_beyond_its_array(env):
    torch, binding = env
    w = eg.WORKLOADS["pileup_100k"]
    dev = torch.device("cuda", 0)
    x = torch.zeros(4, device=dev)
    lay = torch.zeros(4, dtype=torch.uint8, device=dev)
    acc = torch.zeros(w.binning.n_qpt * w.binning.n_phi, dtype=torch.int16, device=dev)
    with pytest.raises(binding.HoughError) as e:
        binding.vote_static(w.geometry, w.binning, x, x, x, lay, (1 << 17) + 1, acc)
    assert e.value.code == binding.ECAPACITY and b"131072" in binding.load().hough_last_error()
    big = eg.with_binning(w, n_phi=8192).binning
    with pytest.raises(binding.HoughError) as e:
        binding.vote_static(w.geometry, big, x, x, x, lay, 4, acc)
    assert e.value.code == binding.ECAPACITY


def test_static_vote_many_rows_and_non_uniform_radii(env):
    # every vote takes the per-vote path (FP32 arcsine, FP64 near an edge), whose inputs include the
    # q/pT centres the entry point computes on the device: they must round like a context's
    torch, binding = env
    w = eg.with_binning(eg.WORKLOADS["pileup_100k"], n_qpt=1024)
    ev = w.event(7).subset(np.arange(20000))
    ev.r = (ev.r + np.random.default_rng(3).uniform(-0.5, 0.5, ev.n_hits)).astype(np.float32)
    got, err = _static_accumulator(torch, binding, w, ev)
    assert err == 0
    assert np.array_equal(got, _context_accumulator(binding, w, ev))


def test_static_vote_allocates_nothing_after_the_first_call(env):
    torch, binding = env
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    pileup, small = eg.WORKLOADS["pileup_100k"], eg.WORKLOADS["single_50trk"]
    cases = []
    for w, ev in ((pileup, pileup.event(2)), (small, small.event(3))):
        hits = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (ev.r, ev.phi, ev.z, ev.layer)]
        acc = torch.empty((w.binning.n_qpt, w.binning.n_phi), dtype=torch.int16, device=dev)
        err = torch.zeros((1,), dtype=torch.int32, device=dev)
        cases.append((w, ev, hits, acc, err))

    def run_all():
        for w, ev, hits, acc, err in cases:
            binding.vote_static(w.geometry, w.binning, *hits, ev.n_hits, acc, err, stream=stream)

    run_all()   # the first calls load the library's device code (and reserve its array) if not yet done
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info(dev)[0], torch.cuda.memory_allocated(dev)
    for _ in range(3):
        run_all()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    assert torch.cuda.memory_allocated(dev) == alloc0
    for w, ev, hits, acc, err in cases:
        assert int(err.item()) == 0
        assert np.array_equal(acc.cpu().numpy().view(np.uint16), _context_accumulator(binding, w, ev))


def test_static_vote_rejects_a_misaligned_accumulator(env):
    torch, binding = env
    w = eg.WORKLOADS["single_50trk"]
    dev = torch.device("cuda", 0)
    x = torch.ones(4, device=dev)
    lay = torch.zeros(4, dtype=torch.uint8, device=dev)
    acc = torch.zeros(w.binning.n_qpt * w.binning.n_phi + 8, dtype=torch.int16, device=dev)
    with pytest.raises(binding.HoughError) as e:
        binding.vote_static(w.geometry, w.binning, x, x, x, lay, 4, acc[1:])   # 2 bytes past an aligned start
    assert e.value.code == binding.EINVAL and b"16-byte" in binding.load().hough_last_error()
