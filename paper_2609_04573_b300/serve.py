"""Serving loop for progressive retrieval (continuous batching).

Refactored fields stay resident on the device (their handles own the plane
streams).  Requests -- (field, target[, box]) -- arrive at any time; a worker
thread admits them while the memory the in-flight retrievals need (output +
scratch, from pcr_retrieve_scratch_bytes) stays under a budget, groups the
admitted requests into one pcr_retrieve_batch_plan call (one decode work list for
the whole group), and keeps up to `streams` groups on the GPU at once on
separate CUDA streams.  Requests that arrive while groups are running join the
next group as soon as memory frees up; results complete out of order through
CUDA events.  Every result is the same field a single retrieval of that
request produces (the kernels are deterministic and share no state between
requests).

Box requests are retrieved with pcr_retrieve_box on the group's stream: only
the box's dependency region is decoded and reconstructed, and the result is
the box of the whole-field retrieval under the same plan.

A request can be cancelled (Request.cancel) until its group is launched: it
is then dropped from the group, its memory is not charged and its future
stays cancelled.  A request whose plan fails gets the exception on its
future; the rest of its group runs.
"""
import queue
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field
from typing import Optional, Tuple

import torch

from . import Target, retrieve_batch


@dataclass
class Request:
    field_id: int
    target: Target
    box: Optional[Tuple[Tuple[int, int], ...]] = None   # ((lo, hi), ...) per axis
    t_submit: float = 0.0
    t_done: float = 0.0
    future: Future = field(default_factory=Future)
    plan: object = None
    bytes_read: int = 0

    @property
    def latency(self):
        return self.t_done - self.t_submit

    def cancel(self):
        """True if the request will not run (cancelled before its launch)."""
        return self.future.cancel()


class Server:
    """Continuous-batching retrieval server over resident handles."""

    def __init__(self, handles, mem_budget=8 << 30, max_batch=32, streams=2, device=None, start=True):
        self.handles = list(handles)
        self.budget = int(mem_budget)
        self.max_batch = max_batch
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self.q = queue.Queue()
        self.inflight = []            # (event, stream, [requests], [outs], mem)
        self.mem_in_use = 0
        self.done = []
        self._stop = False
        self._need = [h.retrieve_scratch_bytes() + h.out_bytes for h in self.handles]
        # a box retrieval reconstructs into a field-sized buffer before copying the box
        self._worker = threading.Thread(target=self._run, daemon=True)
        self.batches = 0
        self.cancelled = 0
        if start:
            self._worker.start()

    def start(self):
        """Start the worker of a server made with start=False (requests
        submitted before then wait in the queue and are batched together)."""
        if self._worker.ident is None:
            self._worker.start()

    def submit(self, field_id, target, box=None):
        r = Request(field_id, target, box, t_submit=time.perf_counter())
        self.q.put(r)
        return r

    def close(self):
        self._stop = True
        if self._worker.ident is None:   # never started: serve what is queued, then stop
            self._worker.start()
        self._worker.join()

    # ---- worker -----------------------------------------------------------
    def _run(self):
        torch.cuda.set_device(self.device)
        pending = []
        sidx = 0
        while True:
            try:
                while True:
                    pending.append(self.q.get_nowait())
            except queue.Empty:
                pass
            self._poll()
            if self._stop and not pending and not self.inflight and self.q.empty():
                return
            free_stream = len(self.inflight) < len(self.streams)
            if pending and free_stream:
                group, mem = [], 0
                rest = []
                for r in pending:
                    need = self._need_of(r)
                    if len(group) < self.max_batch and self.mem_in_use + mem + need <= self.budget:
                        group.append(r)
                        mem += need
                    else:
                        rest.append(r)
                if not group and not self.inflight and pending:
                    # a single request larger than the budget runs alone
                    group, rest = [pending[0]], pending[1:]
                    mem = self._need_of(pending[0])
                pending = rest
                if group:
                    self._launch(group, mem, self.streams[sidx % len(self.streams)])
                    sidx += 1
                    continue
            time.sleep(0.0002)

    def _need_of(self, r):
        n = self._need[r.field_id]
        if r.box is not None:
            h = self.handles[r.field_id]
            n += h.out_bytes   # the field-sized reconstruction buffer of the box path
        return n

    def _launch(self, group, mem, stream):
        hs, plans, outs, boxes = [], [], [], []
        live = []
        for r in group:
            if not r.future.set_running_or_notify_cancel():   # cancelled while queued
                self.cancelled += 1
                continue
            h = self.handles[r.field_id]
            try:
                p = h.plan(r.target, allow_unsat=True)
            except Exception as e:  # isolate a failed request, keep the others
                r.t_done = time.perf_counter()
                r.future.set_exception(e)
                continue
            r.plan = p
            r.bytes_read = p.bytes
            live.append(r)
            if r.box is None:
                hs.append(h)
                plans.append(p)
                with torch.cuda.stream(stream):
                    outs.append(torch.empty(h.shape, dtype=h.dtype, device=self.device))
            else:
                boxes.append((r, h, p))
        if not live:
            return
        mem = sum(self._need_of(r) for r in live)   # the requests that run
        with torch.cuda.stream(stream):
            if hs:
                retrieve_batch(hs, plans, outs, stream=stream)
            res = {}
            for r, h, p in boxes:
                res[id(r)] = h.retrieve_box(p, r.box, stream=stream)[0]
            it = iter(outs)
            results = [res[id(r)] if r.box is not None else next(it) for r in live]
            ev = torch.cuda.Event()
            ev.record(stream)
        self.mem_in_use += mem
        self.inflight.append((ev, stream, live, results, mem))
        self.batches += 1

    def _poll(self):
        keep = []
        for ev, stream, reqs, outs, mem in self.inflight:
            if ev.query():
                now = time.perf_counter()
                for r, o in zip(reqs, outs):
                    r.t_done = now
                    r.future.set_result(o)
                    self.done.append(r)
                self.mem_in_use -= mem
            else:
                keep.append((ev, stream, reqs, outs, mem))
        self.inflight = keep


def percentile(xs, p):
    if not xs:
        return None
    s = sorted(xs)
    k = min(len(s) - 1, max(0, int(round(p / 100.0 * (len(s) - 1)))))
    return s[k]
