"""Serving many graphs on one GPU with continuous batching and admission by device memory.

Sessions (one graph each) open, receive edge-update requests and close. The scheduler
(host logic only, engine-agnostic) decides:

* admission: a session's graph is admitted when its device footprint (damf_bytes_required)
  fits in what the budget has left; sessions wait in first-come order (the head waits for
  room, so a large graph is not starved by smaller ones behind it);
* steps: each step takes at most one request, the oldest, from every resident session with
  requests waiting, so that a graph receives its requests one batch per request, in arrival
  order, exactly as it would alone; the step's graphs run together on the device;
* continuous batching: requests that arrive while steps are on the device join the next step;
  up to `run_ahead` steps are in flight at once, and sessions are admitted and released
  between steps as memory frees up;
* release: a closed session's memory returns to the budget once every step it took part in
  has completed;
* eviction: when the first waiting session does not fit, resident sessions that are idle (no
  request waiting or running) are evicted, least recently active first, if that makes room:
  their graph is checkpointed to host memory and freed, and a request for an evicted session
  puts it back in the admission queue, where it is restored from the checkpoint (the restored
  graph continues exactly where it stopped).

The Server couples the scheduler to the library: each admitted graph is a DamfGraph, built on
a worker thread and its own stream so that the loop keeps serving the resident graphs while it
initialises; each step is one damf_fleet_step over the resident graphs (graphs without a
request take an empty batch), its events copied from pinned host memory in one transfer.
"""

from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import time
from typing import Deque, Dict, List, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    sid: int
    src: np.ndarray
    dst: np.ndarray
    op: np.ndarray
    t_arrive: float
    t_issue: Optional[float] = None
    t_done: Optional[float] = None
    step: Optional[int] = None
    resident_at_arrival: Optional[bool] = None

    @property
    def k(self) -> int:
        return int(self.src.shape[0])


@dataclasses.dataclass
class Session:
    sid: int
    nbytes: int
    state: str = "waiting"          # waiting -> admitting -> resident -> released -> freed;
                                    # resident -> evicting -> evicted -> waiting (readmission)
    queue: Deque[Request] = dataclasses.field(default_factory=collections.deque)
    closing: bool = False
    last_step: int = -1             # the latest step that holds one of its requests
    t_open: float = 0.0
    t_admit: Optional[float] = None
    t_active: float = 0.0           # the latest arrival of one of its requests
    evictions: int = 0


class Scheduler:
    """Admission, per-step request selection and release (no device work)."""

    def __init__(self, budget_bytes: int, max_events: int = 1024, min_idle_s: float = 0.0):
        self.min_idle_s = float(min_idle_s)   # a graph idle for less is not evicted
        self.budget = int(budget_bytes)
        self.used = 0
        self.max_events = int(max_events)
        self.sessions: Dict[int, Session] = {}
        self.waiting: Deque[int] = collections.deque()
        self.next_step_id = 0
        self.done_upto = -1             # every step <= done_upto has completed

    # -- sessions
    def open(self, sid: int, nbytes: int, t: float = 0.0):
        if sid in self.sessions:
            raise ValueError("session %d exists" % sid)
        if nbytes > self.budget:
            raise ValueError("session %d needs %d bytes, more than the whole budget" % (sid, nbytes))
        self.sessions[sid] = Session(sid, int(nbytes), t_open=t)
        self.waiting.append(sid)

    def close(self, sid: int):
        """The session takes no more requests; it is released once its queue is served."""
        self.sessions[sid].closing = True

    def submit(self, req: Request):
        s = self.sessions[req.sid]
        if s.closing:
            raise ValueError("session %d is closing" % req.sid)
        if req.k > self.max_events:
            raise ValueError("request of %d events; at most %d" % (req.k, self.max_events))
        req.resident_at_arrival = s.state == "resident"
        s.queue.append(req)
        s.t_active = max(s.t_active, req.t_arrive)
        if s.state == "evicted":        # readmission: back in the admission queue
            s.state = "waiting"
            self.waiting.append(s.sid)

    def plan_evictions(self, t: float = 0.0) -> List[int]:
        """Idle resident sessions (no request waiting or in a running step, not closing, no
        request for min_idle_s up to time t) to evict, least recently active first, so that
        the first waiting session fits; none when it fits already or when evicting every idle
        session would not make room."""
        if not self.waiting:
            return []
        on_the_way = sum(s.nbytes for s in self.sessions.values() if s.state == "evicting")
        need = self.sessions[self.waiting[0]].nbytes - (self.budget - self.used) - on_the_way
        if need <= 0:
            return []
        idle = sorted((s for s in self.sessions.values()
                       if s.state == "resident" and not s.closing and not s.queue and s.last_step <= self.done_upto
                       and (self.min_idle_s <= 0.0 or t - s.t_active >= self.min_idle_s)),
                      key=lambda s: (s.t_active, s.sid))
        out, freed = [], 0
        for s in idle:
            if freed >= need:
                break
            out.append(s.sid)
            freed += s.nbytes
        return out if freed >= need else []

    def evicting(self, sid: int):
        """The session leaves the device (it takes no further step)."""
        s = self.sessions[sid]
        if s.state != "resident":
            raise ValueError("session %d is not resident" % sid)
        s.state = "evicting"

    def evicted(self, sid: int):
        """Its graph is checkpointed and freed: the memory returns to the budget; with requests
        waiting it is queued for readmission at once."""
        s = self.sessions[sid]
        if s.state != "evicting":
            raise ValueError("session %d is not being evicted" % sid)
        s.state = "evicted"
        s.evictions += 1
        self.used -= s.nbytes
        if s.queue:
            s.state = "waiting"
            self.waiting.append(sid)

    def admissions(self, t: float = 0.0) -> List[int]:
        """Sessions to bring onto the device now (first come, while they fit)."""
        out = []
        while self.waiting:
            s = self.sessions[self.waiting[0]]
            if self.used + s.nbytes > self.budget:
                break
            self.waiting.popleft()
            self.used += s.nbytes
            s.state = "admitting"
            s.t_admit = t
            out.append(s.sid)
        return out

    def admitted(self, sid: int):
        self.sessions[sid].state = "resident"

    def resident(self) -> List[int]:
        return sorted(s.sid for s in self.sessions.values() if s.state == "resident")

    # -- steps
    def next_step(self, t: float = 0.0):
        """(step id, {sid: Request}) with the oldest request of every resident session that has
        one, or None when no resident session has a request waiting."""
        pick = {}
        for sid in self.resident():
            s = self.sessions[sid]
            if s.queue:
                pick[sid] = s.queue.popleft()
        if not pick:
            return None
        step = self.next_step_id
        self.next_step_id += 1
        for sid, r in pick.items():
            r.step, r.t_issue = step, t
            self.sessions[sid].last_step = step
        return step, pick

    def step_done(self, step: int, reqs: Dict[int, Request], t: float):
        """Marks a step complete (steps complete in issue order)."""
        for r in reqs.values():
            r.t_done = t
        self.done_upto = max(self.done_upto, step)

    def releases(self) -> List[int]:
        """Sessions to release now: closing, served, and with none of their requests still
        running. A released session takes no further step; its memory returns to the budget at
        freed(). An evicted session that closes is released at once (nothing is on the device)."""
        out = []
        for s in self.sessions.values():
            if s.state == "resident" and s.closing and not s.queue and s.last_step <= self.done_upto:
                s.state = "released"
                out.append(s.sid)
            elif s.state == "evicted" and s.closing and not s.queue:
                s.state = "freed"
        return out

    def freed(self, sid: int):
        """The released session's device memory is free again."""
        s = self.sessions[sid]
        if s.state != "released":
            raise ValueError("session %d is not released" % sid)
        s.state = "freed"
        self.used -= s.nbytes

    def idle(self) -> bool:
        """No session waits for admission and no resident one has a request waiting."""
        return not self.waiting and all(not s.queue for s in self.sessions.values() if s.state == "resident")

    def backlog(self) -> int:
        """Requests waiting (in resident and in waiting sessions)."""
        return sum(len(s.queue) for s in self.sessions.values())


class Server:
    """Scheduler + library: graphs as DamfGraphs, steps as fleet steps on one stream."""

    def __init__(self, budget_bytes: int, max_events: int = 1024, run_ahead: int = 2, stream=None,
                 on_release=None, share_exponent: float = 1.0, evict: bool = True, min_idle_s: float = 0.0):
        import torch
        self.torch = torch
        self.on_release = on_release   # called (sid, graph) after a released graph's last step, or
        #                                (sid, checkpoint) for a session that closes while evicted
        self.evict = bool(evict)
        self.evicting = []         # (sid, graph, last step it took part in)
        self.saving = {}           # sid -> future of its checkpoint (worker thread)
        self.checkpoints = {}      # sid -> checkpoint of an evicted session (host memory)
        self.share_exponent = float(share_exponent)   # push CTAs ~ (d (n + m))^exponent per graph
        self.sched = Scheduler(budget_bytes, max_events, min_idle_s)
        self.max_events = int(max_events)
        self.run_ahead = int(run_ahead)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.specs = {}            # sid -> (indptr, indices, cfg, omega)
        self.graphs = {}           # sid -> DamfGraph
        self.fleet = None
        self.fleet_sids: List[int] = []
        self.retired = []          # (fleet, last step it served)
        self.to_destroy = []       # (sid, graph, last step it took part in)
        self.inflight = collections.deque()   # (step, reqs, event, buffers)
        self.completed: List[Request] = []
        self.t0 = time.perf_counter()
        self.steps_issued = 0
        self.kernels = 0           # kernels of graphs and fleets already closed
        self.init_pool = concurrent.futures.ThreadPoolExecutor(max_workers=1)
        self.init_stream = torch.cuda.Stream()   # initialisations, restores and checkpoints
        self.initializing = {}     # sid -> future of its DamfGraph
        self.ring = []             # staging buffers (pinned host, device), reused round robin
        self.ring_rows = 0
        self.ring_pos = 0

    def now(self) -> float:
        return time.perf_counter() - self.t0

    # -- client side
    def open(self, sid: int, indptr, indices, cfg, omega):
        from .api import bytes_required
        self.specs[sid] = (indptr, indices, cfg, omega)
        self.sched.open(sid, bytes_required(cfg), self.now())

    def submit(self, rid: int, sid: int, src, dst, op, t_arrive: Optional[float] = None):
        r = Request(rid, sid, np.ascontiguousarray(src, np.int32), np.ascontiguousarray(dst, np.int32),
                    np.ascontiguousarray(op, np.int8), self.now() if t_arrive is None else t_arrive)
        self.sched.submit(r)
        return r

    def close(self, sid: int):
        self.sched.close(sid)

    # -- server loop
    def _rebuild_fleet(self):
        from .api import DamfFleet
        sids = self.sched.resident()
        if sids == self.fleet_sids:   # resident() drops released sessions, so they leave the fleet
            return
        if self.fleet is not None:
            self.retired.append((self.fleet, self.sched.next_step_id - 1))
            self.kernels += self.fleet.launches
        self.fleet = DamfFleet([self.graphs[s] for s in sids]) if sids else None
        if self.fleet is not None and self.share_exponent != 1.0:
            self.fleet.set_shares(exponent=self.share_exponent)
        self.fleet_sids = sids

    def _build(self, spec, ckpt):
        # worker thread: the graph's initialisation (or its restore from an eviction's checkpoint)
        # on its own stream (the library synchronises that stream before returning), beside the
        # steps the loop keeps issuing
        from .api import DamfGraph
        torch = self.torch
        with torch.cuda.stream(self.init_stream):
            if ckpt is not None:
                dev = dict(ckpt, state={k: v.to("cuda", non_blocking=True) for k, v in ckpt["state"].items()})
                g = DamfGraph.restore(dev, stream=self.init_stream)
            else:
                g = DamfGraph(*spec, stream=self.init_stream)
            self.init_stream.synchronize()
        return g

    def _checkpoint(self, g):
        """The graph's checkpoint with its tensors in pinned host memory."""
        ck = g.save()
        torch = self.torch
        # one device-to-host copy per tensor, straight into pinned memory (ordered after the
        # save on the current stream; a copy into host memory returns when it is done)
        ck["state"] = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True).copy_(v)
                       for k, v in ck["state"].items()}
        return ck

    def _evict_job(self, g):
        # worker thread: the checkpoint (its copies and the adjacency export wait for the device
        # there, not in the loop) and the free; returns (checkpoint, kernels the graph launched)
        torch = self.torch
        with torch.cuda.stream(self.init_stream):
            g.check()
            ck = self._checkpoint(g)
            kernels = g.stats()["launches"]
            g.close()
        return ck, kernels

    def _admit(self, block: bool = False):
        if self.evict:
            for sid in self.sched.plan_evictions(self.now()):
                self.sched.evicting(sid)
                # it takes part (empty batch) in every step issued so far
                self.evicting.append((sid, self.graphs.pop(sid), self.sched.next_step_id - 1))
        for sid in self.sched.admissions(self.now()):
            self.initializing[sid] = self.init_pool.submit(self._build, self.specs.pop(sid, None),
                                                           self.checkpoints.pop(sid, None))
        for sid, fut in list(self.initializing.items()):
            if block or fut.done():
                self.graphs[sid] = fut.result()
                del self.initializing[sid]
                self.sched.admitted(sid)

    def wait_admissions(self):
        """Blocks until every graph being initialised is resident."""
        self._admit(block=True)

    def _issue(self) -> bool:
        torch = self.torch
        nxt = self.sched.next_step(self.now())
        if nxt is None:
            return False
        step, reqs = nxt
        self._rebuild_fleet()
        G, K = len(self.fleet_sids), self.max_events
        if G > self.ring_rows:
            # larger staging; in-flight steps keep the old buffers alive through their records
            self.ring_rows = max(G, 2 * self.ring_rows)
            self.ring = [(torch.empty((self.ring_rows, 2 * K + K // 4), dtype=torch.int32).pin_memory(),
                          torch.empty((self.ring_rows, 2 * K + K // 4), dtype=torch.int32, device="cuda"))
                         for _ in range(self.run_ahead + 1)]
        host, dev = self.ring[self.ring_pos]
        self.ring_pos = (self.ring_pos + 1) % len(self.ring)
        hv = host.numpy()
        counts = []
        for i, sid in enumerate(self.fleet_sids):
            r = reqs.get(sid)
            k = r.k if r is not None else 0
            if k:
                hv[i, :k] = r.src
                hv[i, K:K + k] = r.dst
                hv[i, 2 * K:].view(np.int8)[:k] = r.op
            counts.append(k)
        with torch.cuda.stream(self.stream):
            dev[:G].copy_(host[:G], non_blocking=True)
            batches = []
            for i in range(G):
                row = dev[i]
                batches.append((row[:counts[i]], row[K:K + counts[i]], row[2 * K:].view(torch.int8)[:counts[i]]))
            self.fleet.step(batches, self.stream)
            ev = torch.cuda.Event()
            ev.record(self.stream)
        self.inflight.append((step, reqs, ev, (host, dev, batches)))
        self.steps_issued += 1
        return True

    def _retire(self, block: bool):
        while self.inflight:
            step, reqs, ev, _ = self.inflight[0]
            if block:
                ev.synchronize()
            elif not ev.query():
                break
            self.inflight.popleft()
            self.sched.step_done(step, reqs, self.now())
            self.completed.extend(reqs.values())
        for sid in self.sched.releases():
            # it took part (empty batch) in every step issued so far
            self.to_destroy.append((sid, self.graphs.pop(sid), self.sched.next_step_id - 1))
        for sid, s in self.sched.sessions.items():   # sessions that closed while evicted
            if s.state == "freed" and sid in self.checkpoints:
                ck = self.checkpoints.pop(sid)
                if self.on_release is not None:
                    self.on_release(sid, ck)
        done = self.sched.done_upto
        keep = []
        for sid, g, last in self.evicting:
            if last <= done:
                self.saving[sid] = self.init_pool.submit(self._evict_job, g)
            else:
                keep.append((sid, g, last))
        self.evicting = keep
        for sid, fut in list(self.saving.items()):
            if block or fut.done():
                ck, kernels = fut.result()
                self.checkpoints[sid] = ck
                self.kernels += kernels
                del self.saving[sid]
                self.sched.evicted(sid)
        keep = []
        for f, last in self.retired:
            if last <= done:
                f.close()
            else:
                keep.append((f, last))
        self.retired = keep
        keep = []
        for sid, g, last in self.to_destroy:
            if last <= done:
                g.check()
                if self.on_release is not None:
                    self.on_release(sid, g)
                self.kernels += g.stats()["launches"]
                g.close()
                self.sched.freed(sid)
            else:
                keep.append((sid, g, last))
        self.to_destroy = keep

    def poll(self, block: bool = False) -> bool:
        """One turn of the loop: retire finished steps (releasing memory), admit, and issue a
        step when fewer than run_ahead are in flight. Returns whether it issued."""
        self._retire(block=False)
        self._admit()
        issued = False
        if len(self.inflight) < self.run_ahead:
            issued = self._issue()
        if block and not issued and self.inflight:
            self._retire(block=True)
        return issued

    def drain(self, max_seconds: float = float("inf")) -> bool:
        """Serves until nothing more can happen: no step in flight, none to issue, no release or
        admission pending (a session that waits for memory held by sessions that stay open keeps
        waiting). Returns False when max_seconds ran out first."""
        t_end = time.perf_counter() + max_seconds
        while time.perf_counter() < t_end:
            self._retire(block=False)
            self._admit()
            if len(self.inflight) < self.run_ahead and self._issue():
                continue
            if self.inflight or self.to_destroy or self.evicting or self.saving:
                self._retire(block=True)
                continue
            if self.initializing:
                self._admit(block=True)
                continue
            return True
        return False

    def graph(self, sid: int):
        return self.graphs.get(sid)

    def kernel_count(self) -> int:
        """Kernels launched by every graph (initialisation included) and fleet so far."""
        live = sum(g.stats()["launches"] for g in self.graphs.values())
        live += sum(g.stats()["launches"] for _, g, _ in self.to_destroy)
        live += sum(g.stats()["launches"] for _, g, _ in self.evicting)
        return self.kernels + live + (self.fleet.launches if self.fleet is not None else 0)

    def shutdown(self, max_seconds: float = 600.0):
        self.drain(max_seconds)
        self._admit(block=True)
        self.init_pool.shutdown(wait=True)
        self.torch.cuda.synchronize()
        if self.fleet is not None:
            self.fleet.close()
            self.fleet = None
        for f, _ in self.retired:
            f.close()
        self.retired = []
        for sid, g, _ in self.to_destroy:
            if self.on_release is not None:
                self.on_release(sid, g)
            g.close()
            self.sched.freed(sid)
        self.to_destroy = []
        for sid, g, _ in self.evicting:
            self.checkpoints[sid] = self._checkpoint(g)
            g.close()
            self.sched.evicted(sid)
        self.evicting = []
        for sid, fut in list(self.saving.items()):
            self.checkpoints[sid], _ = fut.result()
            self.sched.evicted(sid)
        self.saving = {}
        for g in self.graphs.values():
            g.close()
        self.graphs = {}
