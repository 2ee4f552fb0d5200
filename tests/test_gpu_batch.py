"""Batched processing (needs a GPU): many events of uneven size in one replayed launch sequence.

Each event's accumulator and candidate list in a batch must equal what the single-event path
gives for it alone, bit for bit, and sampled events must match the oracle under the parity rule.
"""
import numpy as np
import pytest

import oracle
from paper_1310_7556_gb300 import eventgen as eg

from parity import (assert_accumulator_parity, assert_candidate_parity)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1310_7556_gb300 import binding as b
    b.load()
    return b


def _alone(binding, w, ev):
    with binding.HoughContext(w.geometry, w.binning, max_hits=max(ev.n_hits, 1), max_candidates=1 << 17,
                              max_members=1 << 21) as ctx:
        ctx.vote_event(ev)
        ctx.peaks()
        ctx.stage2()
        return ctx.accumulator(), ctx.candidates(), ctx.stats()


def _mixed_events():
    w = eg.WORKLOADS["batch_256"]
    evs = [w.event(i) for i in range(12)]
    empty = eg.Event(np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(0, np.float32),
                     np.zeros(0, np.uint8), np.zeros(0, np.int32))
    tiny = w.event(2).subset(np.arange(7))
    return w, evs[:5] + [empty] + evs[5:9] + [tiny] + evs[9:]


def test_batch_equals_events_alone(binding):
    w, events = _mixed_events()
    total = sum(e.n_hits for e in events)
    with binding.HoughBatch(w.geometry, w.binning, max_events=len(events), max_hits=total) as b:
        b.run_events(events)
        cands, offs = b.candidates()
        for e, ev in enumerate(events):
            M_alone, c_alone, st_alone = _alone(binding, w, ev)
            assert np.array_equal(b.accumulator(e), M_alone), f"event {e}"
            assert np.array_equal(cands[offs[e]:offs[e + 1]], c_alone), f"event {e}"
            st = b.stats(e)
            assert st.votes == st_alone.votes and st.n_members == st_alone.n_members
            assert st.stage2_votes == st_alone.stage2_votes


def test_batch_matches_oracle_on_sampled_events(binding):
    """Three events of the batch workload (sparse, tens of thousands of candidates, saturated)
    against the oracle, cell by cell and candidate by candidate."""
    w = eg.WORKLOADS["batch_256"]
    events = [w.event(i) for i in (2, 3, 6)]
    total = sum(e.n_hits for e in events)
    with binding.HoughBatch(w.geometry, w.binning, max_events=3, max_hits=total) as b:
        b.run_events(events)
        cands, offs = b.candidates()
        for e, ev in enumerate(events):
            ref = oracle.run(w.geometry, w.binning, ev)
            assert_accumulator_parity(b.accumulator(e), ref["M"], ref["vote_flags"])
            assert_candidate_parity(cands[offs[e]:offs[e + 1]], ref["candidates"], ref["vote_flags"], w.binning.n_phi)
            assert int(b.stats(e).votes) == int(ref["votes_by_layer"].sum())
            # stage 2 of every candidate whose members and z0 votes the oracle does not flag
            c_gpu = cands[offs[e]:offs[e + 1]]
            key_ref = {(int(c["iq"]), int(c["jphi"])): q for q, c in enumerate(ref["candidates"])}
            mflag = {int(f["cand"]) for f in ref["member_flags"]} | {int(f["cand"]) for f in ref["stage2_flags"]}
            checked = 0
            for c in c_gpu:
                q = key_ref.get((int(c["iq"]), int(c["jphi"])))
                if q is None or q in mflag:
                    continue
                s2 = ref["stage2"][q]
                n_ref = int(ref["member_offsets"][q + 1] - ref["member_offsets"][q])
                assert int(c["n_members"]) == n_ref
                assert (int(c["icot"]), int(c["jz0"]), int(c["mask2"])) == (int(s2["icot"]), int(s2["jz0"]), int(s2["mask2"]))
                checked += 1
            assert checked > 0


def test_graph_replay_on_new_inputs_and_device_pointers(binding):
    """The captured graph is reused for a second batch of the same size with other events, and
    device-resident inputs give the same result as host inputs."""
    import torch
    w = eg.WORKLOADS["batch_256"]
    first = [w.event(i) for i in (0, 2, 7)]
    second = [w.event(i) for i in (4, 5, 2)]
    total = max(sum(e.n_hits for e in first), sum(e.n_hits for e in second))
    with binding.HoughBatch(w.geometry, w.binning, max_events=3, max_hits=total) as b:
        b.run_events(first)
        b.run_events(second)
        cands, offs = b.candidates()
        for e, ev in enumerate(second):
            M_alone, c_alone, _ = _alone(binding, w, ev)
            assert np.array_equal(b.accumulator(e), M_alone)
            assert np.array_equal(cands[offs[e]:offs[e + 1]], c_alone)
        hs = np.zeros(4, np.int64)
        hs[1:] = np.cumsum([e.n_hits for e in second])
        dev = [torch.from_numpy(np.concatenate([getattr(e, k) for e in second])).cuda() for k in ("r", "phi", "z", "layer")]
        torch.cuda.synchronize()
        b.run(*dev, hs, where=binding.DEVICE)
        cands2, offs2 = b.candidates()
        assert np.array_equal(cands2, cands) and np.array_equal(offs2, offs)


def test_batch_limits(binding):
    w = eg.WORKLOADS["single_50trk"]
    evs = [w.event(i) for i in range(3)]
    with binding.HoughBatch(w.geometry, w.binning, max_events=2, max_hits=10_000) as b:
        with pytest.raises(binding.HoughError) as e:
            b.run_events(evs)
        assert e.value.code == binding.ECAPACITY
    with binding.HoughBatch(w.geometry, w.binning, max_events=4, max_hits=100) as b:
        with pytest.raises(binding.HoughError) as e:
            b.run_events(evs)
        assert e.value.code == binding.ECAPACITY
