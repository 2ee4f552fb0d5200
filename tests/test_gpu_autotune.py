"""The autotuner (needs a GPU): it times a sweep of kernel configurations on a batch, applies the
fastest, and that configuration gives the same results as the default; a cache file makes a second
tuning a lookup."""
import numpy as np
import pytest

from paper_1310_7556_gb300 import eventgen as eg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1310_7556_gb300 import binding as b
    b.load()
    return b


def _batch_inputs():
    w = eg.WORKLOADS["batch_256"]
    rng = np.random.default_rng(5)
    events = []
    for i in range(5):
        ev = w.event(i)
        if ev.n_hits > 15_000:
            ev = ev.subset(np.sort(rng.choice(ev.n_hits, 15_000, replace=False)))
        events.append(ev)
    hs = np.zeros(len(events) + 1, np.int64)
    hs[1:] = np.cumsum([e.n_hits for e in events])
    cat = lambda k, dt: np.concatenate([getattr(e, k) for e in events]).astype(dt)
    return w, (cat("r", np.float32), cat("phi", np.float32), cat("z", np.float32), cat("layer", np.uint8)), hs


def test_autotune_applies_a_configuration_with_identical_results(binding, tmp_path):
    w, hits, hs = _batch_inputs()
    cache = str(tmp_path / "tune.txt")
    with binding.HoughBatch(w.geometry, w.binning, max_events=8, max_hits=int(hs[-1])) as b:
        b.run(*hits, hs)
        ref, ref_offs = b.candidates()
        res = b.autotune(*hits, hs, reps=1, cache_path=cache)
        assert res.from_cache == 0 and res.tried >= 10 and res.ms > 0 and res.default_ms > 0
        assert res.ms <= res.default_ms
        b.run(*hits, hs)
        got, got_offs = b.candidates()
        assert np.array_equal(got, ref) and np.array_equal(got_offs, ref_offs)
        again = b.autotune(*hits, hs, reps=1, cache_path=cache)
        assert again.from_cache == 1
        assert [getattr(again.tiling, f) for f in binding.TILING_FIELDS] == \
               [getattr(res.tiling, f) for f in binding.TILING_FIELDS]
    found = binding.tune_lookup(cache, w.geometry, w.binning, n_events=5)
    assert found == {f: getattr(res.tiling, f) for f in binding.TILING_FIELDS}
    assert binding.tune_lookup(cache, w.geometry, w.binning, n_events=64) is None   # another size bucket
    with open(cache) as f:
        assert len(f.read().strip().splitlines()) == 1
