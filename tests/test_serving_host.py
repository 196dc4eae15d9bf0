"""Host logic of the serving loop (no GPU): first-come-first-served packing
of a call, deadlines that drop a request still waiting for a slot, and
failures that stay with their request unless the whole call failed."""
import collections

import numpy as np
import pytest

from paper_2305_14306_gb300 import hav, serving


class _Pts:
    def __init__(self, n):
        self.shape = (n, 3)


def _req(rid, n, arrival=0.0, deadline=None):
    return serving.Request(rid, arrival, _Pts(n), max(1, n // 4), deadline)


def test_take_batch_is_first_come_first_served_within_the_limits():
    w = collections.deque([_req(0, 100), _req(1, 300), _req(2, 50), _req(3, 10)])
    assert [r.rid for r in serving.take_batch(w, max_segments=8, slot_points=400)] == [0, 1]
    assert [r.rid for r in w] == [2, 3]  # the rest keeps its order
    assert [r.rid for r in serving.take_batch(w, max_segments=1, slot_points=400)] == [2]
    assert [r.rid for r in serving.take_batch(w, max_segments=8, slot_points=5)] == []
    assert [r.rid for r in w] == [3]


def test_large_clouds_are_served_alone_in_arrival_order():
    w = collections.deque([_req(0, 10), _req(1, 20), _req(2, 500), _req(3, 30), _req(4, 600), _req(5, 5)])
    take = lambda: [r.rid for r in serving.take_batch(w, max_segments=8, slot_points=1000, solo_points=400)]
    assert take() == [0, 1]  # a large cloud ends the batch of small ones before it
    assert take() == [2]     # and is a call of its own when it is first in line
    assert take() == [3]
    assert take() == [4]
    assert take() == [5]
    assert take() == [] and not w
    # a large cloud the slot cannot hold is not taken (the server rejects it up front)
    w = collections.deque([_req(0, 2000)])
    assert serving.take_batch(w, max_segments=8, slot_points=1000, solo_points=400) == [] and len(w) == 1
    # without solo_points the same queue packs as before
    w = collections.deque([_req(0, 10), _req(1, 20), _req(2, 500), _req(3, 30)])
    assert [r.rid for r in serving.take_batch(w, max_segments=8, slot_points=1000)] == [0, 1, 2, 3]


def test_expired_requests_are_dropped_before_launch():
    w = collections.deque([_req(0, 10, 0.0, deadline=0.5), _req(1, 10, 0.2), _req(2, 10, 0.4, deadline=0.5),
                           _req(3, 10, 0.1, deadline=0.95)])
    res = {}
    assert serving.expire(w, 1.0, res) == 2
    assert [r.rid for r in w] == [1, 3]
    assert sorted(res) == [0, 2]
    for rid in (0, 2):
        assert res[rid].status == serving.EXPIRED and res[rid].batch == 0 and res[rid].indices.size == 0
    assert abs(res[2].latency - 0.6) < 1e-12
    assert serving.expire(w, 1.0, res) == 0  # no deadline, or not yet passed


def test_a_failed_segment_stays_with_its_request():
    batch = [_req(0, 40), _req(1, 80), _req(2, 20)]
    offsets = np.array([0, 10, 30, 35])
    h_out = np.arange(35, dtype=np.int32)
    res = {}
    serving.collect(batch, offsets, h_out, hav.HAV_ERR_NONFINITE, [0, hav.HAV_ERR_NONFINITE, 0], 1.0, res)
    assert [res[k].status for k in range(3)] == [0, hav.HAV_ERR_NONFINITE, 0]
    assert np.array_equal(res[0].indices, np.arange(10)) and np.array_equal(res[2].indices, np.arange(30, 35))
    assert all(res[k].batch == 3 for k in range(3))


@pytest.mark.parametrize("st", [hav.HAV_ERR_TIMEOUT, hav.HAV_ERR_CUDA, hav.HAV_ERR_INVALID, hav.HAV_ERR_NOMEM])
def test_a_failed_call_stops_the_loop(st):
    with pytest.raises(hav.HavError):
        serving.collect([_req(0, 40)], np.array([0, 10]), np.zeros(10, np.int32), st, [0], 1.0, {})


class _Event:
    def __init__(self, ready_at, clock):
        self.ready_at, self.clock = ready_at, clock

    def query(self):
        return self.clock() >= self.ready_at


class _Host:
    def __init__(self, a):
        self.a = a

    def numpy(self):
        return self.a


class _FakeServer(serving.Server):
    """The real serving loop with the device work replaced: a call 'runs' for
    `busy` seconds of the fake clock and returns each segment's local indices."""

    def __init__(self, clock, slots=2, slot_points=1000, max_segments=4, busy=1.0):
        self.params, self.max_segments, self.slot_points = None, max_segments, slot_points
        self.clock, self.busy, self.calls = clock, busy, []
        self.slots = [serving._Slot(stream=None, ctx=None, d_pts=None, d_out=None, h_out=None)
                      for _ in range(slots)]

    def _launch(self, slot, batch):
        ms = [r.m for r in batch]
        slot.h_out = _Host(np.concatenate([np.arange(m, dtype=np.int32) for m in ms]))
        slot.event = _Event(self.clock() + self.busy, self.clock)
        slot.batch = batch
        slot.offsets = np.concatenate([[0], np.cumsum(ms)])
        self.calls.append([r.rid for r in batch])


def test_the_loop_serves_expires_and_isolates_failures(monkeypatch):
    t = [0.0]

    def clock():  # every reading advances the fake time a little
        t[0] += 0.01
        return t[0]

    bad = {3}
    srv = _FakeServer(clock, slots=1, slot_points=1000, max_segments=2, busy=1.0)

    def status_of_current(ctx, n, stream=None):
        slot = srv.slots[0]
        per = [hav.HAV_ERR_NONFINITE if r.rid in bad else 0 for r in slot.batch]
        return (hav.HAV_ERR_NONFINITE if any(per) else 0), per

    monkeypatch.setattr(hav, "hav_status_get", status_of_current)
    reqs = [_req(0, 40), _req(1, 40), _req(2, 40, 0.0, deadline=0.5), _req(3, 40), _req(4, 40, 0.0, deadline=30.0)]
    res = srv.serve(reqs, clock=clock)
    assert sorted(res) == [0, 1, 2, 3, 4]
    # one slot, two requests a call, each call busy for 1 s: request 2 waits past its deadline
    assert res[2].status == serving.EXPIRED and res[2].batch == 0
    assert 2 not in [rid for call in srv.calls for rid in call]
    assert res[3].status == hav.HAV_ERR_NONFINITE  # its own failure only
    for rid in (0, 1, 4):
        assert res[rid].status == 0 and np.array_equal(res[rid].indices, np.arange(10))
    assert srv.calls[0] == [0, 1]
