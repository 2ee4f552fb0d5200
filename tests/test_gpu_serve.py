"""Served mode (needs a GPU): events submitted one by one, continuously batched by the library's
dispatcher, must give each event the same result as processing it alone, bit for bit, whatever
else shares its launch.  Admission limits and failure handling are exercised with host-side
faults only (a held dispatcher, a stream whose completion is never observed, a failed
allocation): no test faults, traps or hangs the GPU.
"""
import threading
import time

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


W = eg.WORKLOADS["batch_256"]


def _events(n, max_hits=12_000):
    """Events of the batch workload, cut to at most max_hits hits (a random subset), plus an
    empty and a tiny event."""
    rng = np.random.default_rng(7)
    out = []
    for i in range(n):
        ev = W.event(i)
        if ev.n_hits > max_hits:
            ev = ev.subset(np.sort(rng.choice(ev.n_hits, max_hits, replace=False)))
        out.append(ev)
    empty = eg.Event(np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(0, np.float32),
                     np.zeros(0, np.uint8), np.zeros(0, np.int32))
    out.insert(3, empty)
    out.insert(7, W.event(1).subset(np.arange(9)))
    return out


def _alone(binding, ev):
    with binding.HoughContext(W.geometry, W.binning, max_hits=max(ev.n_hits, 1), max_candidates=1 << 17,
                              max_members=1 << 21) as ctx:
        c = ctx.process(ev.r, ev.phi, ev.z, ev.layer, ev.n_hits)
        return c, int(ctx.stats().votes)


def _server(binding, **kw):
    args = dict(max_batch_events=8, max_batch_hits=8 * 12_000, lanes=3, max_candidates=1 << 17,
                max_members=1 << 21)
    args.update(kw)
    return binding.HoughServer(W.geometry, W.binning, **args)


def test_served_results_equal_alone(binding):
    events = _events(22)
    expect = [_alone(binding, ev) for ev in events]
    tickets = [None] * len(events)
    with _server(binding) as srv:
        # part of the stream arrives while launches are held, so batches of several events form;
        # the rest comes from two threads at random times while earlier batches run
        srv.inject(binding.SERVE_FAULT_HOLD, True)
        for i in range(6):
            tickets[i] = srv.submit_event(events[i])
        srv.inject(binding.SERVE_FAULT_HOLD, False)

        def feed(idx, seed):
            rng = np.random.default_rng(seed)
            for i in idx:
                time.sleep(float(rng.uniform(0, 0.002)))
                t = None
                while t is None:      # busy: retry until a lane frees
                    t = srv.submit_event(events[i])
                    if t is None:
                        time.sleep(0.0005)
                tickets[i] = t

        rest = list(range(6, len(events)))
        th = [threading.Thread(target=feed, args=(rest[k::2], 11 + k)) for k in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        sizes = []
        for i, ev in enumerate(events):
            cands, res = srv.poll(tickets[i], timeout_us=30_000_000)
            assert res.status == binding.OK
            c_alone, votes_alone = expect[i]
            assert np.array_equal(cands, c_alone), f"event {i}: served result differs from the event alone"
            assert res.votes == votes_alone
            assert res.arrival_ns <= res.launch_ns <= res.done_ns
            sizes.append(res.batch_events)
        st = srv.stats()
        assert st.completed == len(events) and st.failed == 0 and st.pending_tickets == 0
        assert st.launched_events == len(events)
        assert max(sizes) > 1, "no launch held more than one event"


def test_unpolled_results_fill_the_pool_then_are_copied(binding):
    """Full-size events, four per launch: a batch's candidates overflow the mapped part of its
    result block (16,384 candidates), so polls read across both parts; six batches left unpolled
    hold every block the pool may allocate (three per lane), so the last completions copy their
    events' candidates out instead.  Every event still equals its result alone."""
    base = [W.event(i) for i in range(8)]
    expect = [_alone(binding, ev)[0] for ev in base]
    per = 4
    with _server(binding, lanes=2, max_batch_events=per,
                 max_batch_hits=per * max(ev.n_hits for ev in base)) as srv:
        tickets = []
        for b in range(6):
            srv.inject(binding.SERVE_FAULT_HOLD, True)
            tickets += [srv.submit_event(base[(b * per + k) % len(base)]) for k in range(per)]
            srv.inject(binding.SERVE_FAULT_HOLD, False)
            srv.drain(timeout_us=30_000_000)
        assert all(t is not None for t in tickets)
        assert srv.stats().pending_tickets == len(tickets)
        n_first = 0
        for i, t in enumerate(tickets):
            cands, res = srv.poll(t, timeout_us=30_000_000)
            assert res.status == binding.OK and res.batch_events == per
            assert np.array_equal(cands, expect[i % len(base)]), f"event {i}"
            n_first += res.n_candidates if i < per else 0
        assert n_first > 16_384, "the first batch did not reach into its block's overflow"


def test_admission_is_bounded_and_hold_times_out(binding):
    events = _events(6)
    with _server(binding, max_batch_events=2, lanes=2) as srv:
        srv.inject(binding.SERVE_FAULT_HOLD, True)
        got = [srv.submit_event(events[i]) for i in range(5)]
        assert all(t is not None for t in got[:4]) and got[4] is None, "two lanes of two events admit four"
        st = srv.stats()
        assert st.admitted == 4 and st.rejected_busy == 1
        with pytest.raises(binding.HoughError) as e:
            srv.poll(got[0], timeout_us=20_000)
        assert e.value.code == binding.ETIMEDOUT
        srv.inject(binding.SERVE_FAULT_HOLD, False)
        for i in range(4):
            cands, res = srv.poll(got[i], timeout_us=30_000_000)
            assert np.array_equal(cands, _alone(binding, events[i])[0])
            assert res.batch_events == 2


def test_malformed_event_is_refused_alone(binding):
    ev = _events(1)[0]
    bad = eg.Event(ev.r.copy(), ev.phi.copy(), ev.z.copy(), ev.layer.copy(), ev.track.copy())
    bad.layer[5] = 12   # beyond the 10 layers
    with _server(binding) as srv:
        with pytest.raises(binding.HoughError) as e:
            srv.submit_event(bad)
        assert e.value.code == binding.EINVAL
        t = srv.submit_event(ev)
        cands, res = srv.poll(t, timeout_us=30_000_000)
        assert res.status == binding.OK and np.array_equal(cands, _alone(binding, ev)[0])
        assert srv.stats().rejected_invalid == 1


def test_stalled_stream_is_retired_by_the_watchdog(binding):
    events = _events(3)
    with _server(binding, lane_timeout_us=300_000) as srv:
        srv.inject(binding.SERVE_FAULT_STALL, True)
        t = srv.submit_event(events[0])
        _, res = srv.poll(t, timeout_us=10_000_000, candidates=False, allow=(binding.ETIMEDOUT,))
        assert res is not None and res.status == binding.ETIMEDOUT
        st = srv.stats()
        assert st.timeouts == 1 and st.retired_lanes == 1 and st.lanes == 2
        srv.inject(binding.SERVE_FAULT_STALL, False)
        t = srv.submit_event(events[1])
        cands, res = srv.poll(t, timeout_us=30_000_000)
        assert res.status == binding.OK and np.array_equal(cands, _alone(binding, events[1])[0])


def test_result_allocation_failure_fails_one_batch(binding):
    events = _events(3)
    with _server(binding) as srv:
        srv.inject(binding.SERVE_FAULT_ALLOC, True)
        t = srv.submit_event(events[0])
        _, res = srv.poll(t, timeout_us=30_000_000, candidates=False, allow=(binding.ENOMEM,))
        assert res.status == binding.ENOMEM
        t = srv.submit_event(events[2])
        cands, res = srv.poll(t, timeout_us=30_000_000)
        assert res.status == binding.OK and np.array_equal(cands, _alone(binding, events[2])[0])
        st = srv.stats()
        assert st.alloc_failures == 1 and st.failed == 1 and st.lanes == 3


def test_memory_budget_and_config_checks(binding):
    with pytest.raises(binding.HoughError) as e:
        _server(binding, memory_budget=1 << 20)
    assert e.value.code == binding.ENOMEM
    with pytest.raises(binding.HoughError) as e:
        _server(binding, lanes=1)
    assert e.value.code == binding.EINVAL
    with pytest.raises(binding.HoughError) as e:
        _server(binding, lanes=2, max_in_flight=2)
    assert e.value.code == binding.EINVAL
    # lanes = 0: as many as the budget holds (at most four)
    with _server(binding, lanes=0, max_batch_events=2, max_batch_hits=20_000) as srv:
        st = srv.stats()
        assert 2 <= st.lanes <= 4 and st.device_bytes > 0
        with _server(binding, lanes=0, max_batch_events=2, max_batch_hits=20_000,
                     memory_budget=int(st.device_bytes // st.lanes * 2.5)) as two:
            assert two.stats().lanes == 2


def test_replay_offers_every_arrival_and_polls_every_admitted_event(binding):
    events = _events(4)
    pool = [tuple(np.ascontiguousarray(getattr(e, k)) for k in ("r", "phi", "z", "layer")) for e in events]
    with _server(binding) as srv:
        start = binding.serve_clock_ns() + 20_000_000
        arrival = start + np.arange(40, dtype=np.int64) * 500_000   # 2,000 events/s
        res = srv.replay(pool, arrival, threads=3)
        assert res.shape == (40,)
        admitted = res["ticket"] != 0
        assert admitted.sum() >= 1
        assert np.all(res["status"][admitted] == binding.OK)
        assert np.all(res["status"][~admitted] == binding.EBUSY)
        assert np.all(res["arrival_ns"] == arrival)
        assert np.all(res["done_ns"][admitted] >= res["arrival_ns"][admitted])
        # each admitted arrival's vote count is its pool event's
        votes = [_alone(binding, ev)[1] for ev in events]
        for i in np.flatnonzero(admitted):
            assert int(res["votes"][i]) == votes[i % len(pool)]
        st = srv.stats()
        assert st.admitted == admitted.sum() and st.completed == admitted.sum() and st.pending_tickets == 0


@pytest.mark.parametrize("variant", ["counts", "d0"])
def test_served_variants_equal_alone(binding, variant):
    """The count accumulator and the d0 axis through the server: each event as alone."""
    if variant == "counts":
        w = eg.with_binning(W, accumulator=eg.ACC_COUNTS, threshold=12)
        events = _events(10)
    else:
        w = eg.WORKLOADS["displaced_d0"]
        events = [w.event(i) for i in range(8)]
    expect = []
    for ev in events:
        with binding.HoughContext(w.geometry, w.binning, max_hits=max(ev.n_hits, 1), max_candidates=1 << 17,
                                  max_members=1 << 21) as ctx:
            expect.append(ctx.process(ev.r, ev.phi, ev.z, ev.layer, ev.n_hits).copy())
    with binding.HoughServer(w.geometry, w.binning, max_batch_events=4, max_batch_hits=4 * 12_000, lanes=2,
                             max_candidates=1 << 17, max_members=1 << 21) as srv:
        srv.inject(binding.SERVE_FAULT_HOLD, True)
        tickets = [srv.submit_event(ev) for ev in events[:4]]
        srv.inject(binding.SERVE_FAULT_HOLD, False)
        for ev in events[4:]:
            t = None
            while t is None:
                t = srv.submit_event(ev)
                if t is None:
                    time.sleep(0.0005)
            tickets.append(t)
        sizes = []
        for i, t in enumerate(tickets):
            cands, res = srv.poll(t, timeout_us=30_000_000)
            assert res.status == binding.OK
            assert np.array_equal(cands, expect[i]), f"event {i}"
            sizes.append(res.batch_events)
        assert max(sizes) > 1
