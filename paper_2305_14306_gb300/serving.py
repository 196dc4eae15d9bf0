"""Continuous-batching serving loop for the sampler.

Requests (a cloud and its budget m) arrive over time.  The server keeps a
few *slots*; each slot owns a CUDA stream, a libhav context limited to its
share of the SMs and device buffers, so the slots' launches run side by
side on the GPU; requests bring their points in pinned host memory.  Whenever a slot is free, the
requests that have arrived and wait are packed, first come first served,
into one segmented ``hav_sample_batched`` call, as many as fit the slot's
point capacity and segment limit (admission by workspace memory).  With
``solo_points`` set, a cloud of at least that many points is served alone
(a call of one large cloud gets the library's Morton sort and ownership
test, and its latency no longer waits on a batch's longest search); on
GB300 that lowered the p99 latency of the 10k-1M point mix at 0.95 load
from 2.6 to 1.4-1.6 ms but cut throughput from 3.1x to 2.2-2.8x the plain
path, as a batch shares its sequential passes among all its clouds, so
it is off by default.  A
request's points stay on the device from admission to completion; its
latency runs from its arrival to the moment the host sees its slot's
completion event.

The plain per-cloud path is the same loop with one slot and one request per
call.  Either way every request's indices equal a stand-alone call's.

Failures stay with their request.  A request whose cloud the library rejects
(a non-finite coordinate, a key out of range) gets that status in its
result while the other requests of the same call keep their exact indices
(the library contains such errors to their segment); only a failure of the
whole call (a device wait that gave up, a CUDA error) stops the loop.  A
request may carry a deadline: if it is still waiting for a slot that long
after its arrival, it is dropped with the status EXPIRED and never launched.
This module only orchestrates: every step of the sampling runs in libhav's
kernels.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import hav


EXPIRED = -1  # a request dropped before launch: its deadline passed while it waited


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    points: object          # (n, 3) float32 torch tensor in pinned host memory
    m: int                  # budget (one level)
    deadline: float | None = None  # longest wait for a slot (seconds after arrival); None: no limit


@dataclass
class Result:
    indices: np.ndarray
    latency: float          # seconds from arrival to completion seen by the host
    batch: int              # requests in the call that served it (0: never launched)
    status: int = 0         # hav status of the request's segment (HAV_OK), or EXPIRED


# the statuses that void a whole call rather than one segment of it
_CALL_FAILURES = (hav.HAV_ERR_INVALID, hav.HAV_ERR_TIMEOUT, hav.HAV_ERR_NOMEM, hav.HAV_ERR_CUDA)


def expire(waiting, now: float, results: dict) -> int:
    """Drop the waiting requests whose deadline has passed (results get EXPIRED);
    returns how many were dropped.  The others keep their order."""
    keep, dropped = [], 0
    while waiting:
        r = waiting.popleft()
        if r.deadline is not None and now - r.arrival > r.deadline:
            results[r.rid] = Result(np.empty(0, dtype=np.int32), now - r.arrival, 0, EXPIRED)
            dropped += 1
        else:
            keep.append(r)
    waiting.extend(keep)
    return dropped


def take_batch(waiting, max_segments: int, slot_points: int, solo_points: int | None = None) -> list:
    """First come, first served: the waiting requests that fit one call of a
    slot (at most max_segments clouds and slot_points points in total).  With
    solo_points, a cloud of at least that many points goes alone: it is the
    call when it is first in line, and it ends a batch of smaller ones."""
    def solo(r):
        return solo_points is not None and r.points.shape[0] >= solo_points

    if waiting and solo(waiting[0]):
        return [waiting.popleft()] if waiting[0].points.shape[0] <= slot_points else []
    batch, pts = [], 0
    while (waiting and len(batch) < max_segments and not solo(waiting[0])
           and pts + waiting[0].points.shape[0] <= slot_points):
        r = waiting.popleft()
        batch.append(r)
        pts += r.points.shape[0]
    return batch


def collect(batch, offsets, h_out, status: int, per_segment, now: float, results: dict):
    """Results of a finished call: each request its slice of the indices and its
    segment's status; a failure of the whole call raises."""
    if status in _CALL_FAILURES:
        raise hav.HavError(status, "serving batch")
    for k, (r, a, b) in enumerate(zip(batch, offsets[:-1], offsets[1:])):
        results[r.rid] = Result(h_out[a:b].copy(), now - r.arrival, len(batch), int(per_segment[k]))


@dataclass
class _Slot:
    stream: object
    ctx: hav.Context
    d_pts: object           # device float32 (cap, 3)
    d_out: object           # device int32 (cap,)
    h_out: object           # pinned int32 (cap,)
    event: object = None
    batch: list = field(default_factory=list)
    offsets: np.ndarray = None


class Server:
    solo_points = None  # clouds of at least this many points are served alone (None: never)

    def __init__(self, slots: int = 4, slot_points: int = 2_000_000, max_segments: int = 64,
                 params: hav.hav_params | None = None, share_sms: bool = True,
                 solo_points: int | None = None):
        import torch
        self.torch = torch
        self.params = params or hav.params()
        self.max_segments = max_segments
        self.slot_points = slot_points
        self.solo_points = solo_points
        self.slots = []
        for _ in range(slots):
            ctx = hav.Context(slot_points, max_segments)
            self.slots.append(_Slot(
                stream=torch.cuda.Stream(), ctx=ctx,
                d_pts=torch.empty((slot_points, 3), dtype=torch.float32, device="cuda"),
                d_out=torch.empty(slot_points, dtype=torch.int32, device="cuda"),
                h_out=torch.empty(slot_points, dtype=torch.int32).pin_memory()))
        if share_sms and slots > 1:
            # co-resident launches: each slot gets an equal share of the SMs
            full = self._max_blocks()
            for s in self.slots:
                s.ctx.set_blocks(max(1, full // slots))

    def _max_blocks(self):
        props = self.torch.cuda.get_device_properties(self.torch.cuda.current_device())
        return props.multi_processor_count

    def close(self):
        for s in self.slots:
            s.ctx.close()

    # ------------------------------------------------------------------
    def _launch(self, slot: _Slot, batch):
        torch = self.torch
        sizes = np.array([r.points.shape[0] for r in batch], dtype=np.int64)
        offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        ms = np.array([[r.m for r in batch]], dtype=np.int64)
        total, mt = int(offs[-1]), int(ms.sum())
        with torch.cuda.stream(slot.stream):
            for r, a in zip(batch, offs[:-1]):  # pinned host -> the slot's device buffer
                slot.d_pts[int(a):int(a) + r.points.shape[0]].copy_(r.points, non_blocking=True)
            out = slot.d_out[:mt]
            hav.hav_sample_batched(slot.ctx, slot.d_pts[:total], offs, ms, self.params, outs=[out],
                                   stream=slot.stream)
            slot.h_out[:mt].copy_(out, non_blocking=True)
            slot.event = torch.cuda.Event()
            slot.event.record(slot.stream)
        slot.batch = batch
        slot.offsets = np.concatenate([[0], np.cumsum(ms[0])])

    def _finish(self, slot: _Slot, now: float, results: dict):
        st, per = hav.hav_status_get(slot.ctx, len(slot.batch), stream=slot.stream)
        collect(slot.batch, slot.offsets, slot.h_out.numpy(), st, per, now, results)
        slot.batch = []
        slot.event = None

    def serve(self, requests, clock=time.perf_counter) -> dict:
        """Run the requests with their arrival times (real time); returns rid -> Result."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        for r in pending:
            if r.points.shape[0] > self.slot_points:
                raise ValueError(f"request {r.rid} has more points than a slot holds")
        waiting = collections.deque()
        results = {}
        deadlines = any(r.deadline is not None for r in pending)
        t0 = clock()
        while pending or waiting or any(s.batch for s in self.slots):
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            progressed = deadlines and expire(waiting, now, results) > 0
            for s in self.slots:
                if s.batch and s.event.query():
                    self._finish(s, clock() - t0, results)
                    progressed = True
            for s in self.slots:
                if s.batch or not waiting:
                    continue
                self._launch(s, take_batch(waiting, self.max_segments, self.slot_points, self.solo_points))
                progressed = True
            if not progressed:
                time.sleep(20e-6)
        return results


def percentile(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(q * len(xs)))]
