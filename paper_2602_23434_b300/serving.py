"""Continuous-batching server for test-particle tracing requests.

Requests (N particles, S Boris steps, one of several field snapshots that stay
resident on the device) arrive at any time.  Each scheduling round:
  1. admits queued requests in arrival order while their particle state fits
     in the device-memory budget (admission by free HBM); their device
     initialisation (Philox draws, then a cell sort for gather locality) is
     enqueued on the serving stream, with no host synchronisation;
  2. cuts every request with steps left to schedule into work items of
     `chunk` particles that advance min(left, slice_steps) steps;
  3. enqueues the round through the C ABI (the work-list copy and one
     persistent kernel, replayed from a CUDA graph) and records an event.
Two work lists are staged alternately, so round k + 1 is planned and
enqueued while round k runs; the host only waits when both are in flight.
Requests are completed when the event of the round holding their last slice
has passed.  Requests that arrive while others are on the GPU join at the
next round, so their work overlaps on the device with the running ones.  All
arithmetic runs in libpart.so; this module schedules and bookkeeps only.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import time
from dataclasses import dataclass, field

import numpy as np

from . import _lib as P

# int32 cell, f32 off[3], f32 u[6] (the momentum as a compensated pair)
STATE_BYTES_PER_PARTICLE = 4 + 12 + 24

# part_work_item as a numpy record (the layout of include/part.h), so a
# request's work items are written into the pinned work list in one go
ITEM_DTYPE = np.dtype({
    "names": [f[0] for f in P.WorkItem._fields_],
    "formats": ["u8", "u8", "u8", "i8", "i8", "i4", "i4", "i4", "i4", "f8", "f8"],
    "offsets": [getattr(P.WorkItem, f[0]).offset for f in P.WorkItem._fields_],
    "itemsize": C.sizeof(P.WorkItem)})


@dataclass
class Request:
    rid: int
    snapshot: int
    n: int
    steps: int
    seed: int
    q_over_m: float
    dt: float
    u_th: float
    arrival: float
    admitted: float | None = None
    done: float | None = None
    remaining: int = 0        # steps not yet completed on the device
    unplanned: int = 0        # steps not yet put into a round
    cell: object = None
    off: object = None
    u: object = None

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival

    def result(self):
        """(cell, off, u) device tensors once the request is done."""
        if self.done is None:
            raise RuntimeError("request not finished")
        return self.cell, self.off, self.u


@dataclass
class Snapshot:
    part: object          # P.Part in PART_MIXED / PART_BORIS with fields set
    n_cells: tuple
    fields: object


_streams = {}


def serving_stream(torch, device=None):
    """The created (capturable) stream all snapshots and servers of a device use."""
    dev = device or torch.device("cuda", torch.cuda.current_device())
    key = str(dev)
    if key not in _streams:
        _streams[key] = torch.cuda.Stream(device=dev)
    return _streams[key]


def make_snapshot(torch, n: int, seed: int, capacity: int, device=None):
    """Turbulent field snapshot on an n^3 grid (f32, resident), as a mixed
    Boris context able to initialise and sort up to `capacity` particles."""
    from . import synth
    f = synth.em_fields(3, n, seed).reshape(6, -1).astype(np.float32)
    dev = device or torch.device("cuda", torch.cuda.current_device())
    st = serving_stream(torch, dev)
    with torch.cuda.stream(st):
        ft = torch.as_tensor(f).to(dev)
        part = P.Part(P.make_grid(3, n), P.MIXED, P.TSC, P.BORIS, capacity=capacity,
                      stream=st, device=dev)
        part.set_fields(ft)
    st.synchronize()
    return Snapshot(part=part, n_cells=(n, n, n), fields=ft)


class Server:
    """Continuous batching over resident snapshots (see the module docstring).
    keep_results=False releases a request's device state when it completes
    (a long stream then holds only the admitted requests' memory)."""

    PIPELINE = 2          # work lists in flight: round k + 1 is staged while k runs

    def __init__(self, torch, snapshots, mem_budget_bytes: int, max_items: int = 1 << 16,
                 chunk: int = 2048, slice_steps: int = 32, threads: int = 256,
                 ctas_per_sm: int = 4, clock=time.perf_counter, keep_results: bool = True,
                 round_psteps: float | None = None):
        self.torch = torch
        self.L = P.lib()
        self.snaps = snapshots
        self.stream = snapshots[0].part.stream
        self.budget = int(mem_budget_bytes)
        self.chunk = int(chunk)
        self.slice_steps = int(slice_steps)
        self.max_items = int(max_items)
        self.clock = clock
        self.keep_results = keep_results
        # work per round (particle-steps): with a budget, every round gives
        # each request an equal share of it (requests whose whole remaining
        # work fits take all of it), so small requests finish in a round or
        # two; every request still advances at least slice_steps steps per
        # round, so large ones keep their pace.  Without a budget every
        # request advances slice_steps steps per round.
        self.round_psteps = round_psteps
        dbytes, hbytes = C.c_size_t(), C.c_size_t()
        self._check(self.L.part_server_sizes(len(snapshots), max_items, C.byref(dbytes),
                                             C.byref(hbytes)))
        dev = snapshots[0].part.device
        arr = (C.c_void_p * len(snapshots))(*[s.part.ctx.value for s in snapshots])
        self.ws, self.stage, self.hs, self.item_lists, self.item_arrays = [], [], [], [], []
        for _ in range(self.PIPELINE):
            ws = torch.empty(dbytes.value, dtype=torch.uint8, device=dev)
            stage = torch.empty(hbytes.value, dtype=torch.uint8, pin_memory=True)
            h = C.c_void_p()
            self._check(self.L.part_server_init(C.byref(h), arr, len(snapshots), max_items,
                                                C.c_void_p(ws.data_ptr()), dbytes.value,
                                                C.c_void_p(stage.data_ptr()), hbytes.value,
                                                C.c_void_p(self.stream.cuda_stream), threads,
                                                ctas_per_sm))
            self.ws.append(ws)
            self.stage.append(stage)
            self.hs.append(h)
            self.item_lists.append(self.L.part_server_items(h))
            raw = (C.c_char * (max_items * C.sizeof(P.WorkItem))).from_address(
                C.cast(self.item_lists[-1], C.c_void_p).value)
            self.item_arrays.append(np.frombuffer(raw, dtype=ITEM_DTYPE))
        self.h = self.hs[0]
        self.items = self.item_lists[0]
        self.inflight = []        # (event, slot, plan) in enqueue order
        self._slot = 0
        self.queue: list[Request] = []
        self.active: list[Request] = []
        self.finished: list[Request] = []
        self.used = 0
        self.rounds = 0
        self.busy_s = 0.0
        self._busy_from = None
        self.psteps = 0
        self._next = 0

    def _check(self, code):
        if code != 0:
            msg = self.L.part_last_error(None)
            raise P.PartError(code, msg.decode() if msg else "")

    def close(self):
        for h in getattr(self, "hs", []):
            if h is not None and h.value:
                self.L.part_server_sync(h)
                self.L.part_server_destroy(h)
                h.value = None

    # ------------------------------------------------------------------ API
    def submit(self, snapshot: int, n: int, steps: int, seed: int, q_over_m: float = 1.0,
               dt: float | None = None, u_th: float = 0.1, arrival: float | None = None):
        if not (0 <= snapshot < len(self.snaps)):
            raise ValueError("snapshot out of range")
        need = n * STATE_BYTES_PER_PARTICLE
        if need > self.budget:
            raise P.PartError(2, f"request of {n} particles needs {need} B, budget {self.budget} B")
        if n > self.snaps[snapshot].part.capacity:
            raise P.PartError(1, "request larger than the snapshot's initialisation capacity")
        if dt is None:
            g = self.snaps[snapshot].n_cells[0]
            dt = 0.5 * 2.0 / g
        r = Request(self._next, snapshot, int(n), int(steps), int(seed), float(q_over_m),
                    float(dt), float(u_th), self.clock() if arrival is None else arrival)
        r.remaining = r.unplanned = int(steps)
        self._next += 1
        self.queue.append(r)
        return r

    def _admit(self):
        torch = self.torch
        while self.queue:
            r = self.queue[0]
            need = r.n * STATE_BYTES_PER_PARTICLE
            if self.used + need > self.budget:
                break
            self.queue.pop(0)
            dev = self.snaps[r.snapshot].part.device
            with torch.cuda.stream(self.stream):   # allocations belong to the serving stream
                r.cell = torch.empty(r.n, dtype=torch.int32, device=dev)
                r.off = torch.empty((3, r.n), dtype=torch.float32, device=dev)
                r.u = torch.empty((6, r.n), dtype=torch.float32, device=dev)
            sp = self.snaps[r.snapshot].part
            sp.bind(r.n, r.cell, off=r.off, u=r.u)
            sp.init_particles(r.seed, r.u_th)
            sp.sort()
            sp.flush()                     # sorted state into the request's arrays (async)
            self.used += need
            r.admitted = self.clock()
            if r.remaining == 0:
                self._finish(r)
            else:
                self.active.append(r)

    def _finish(self, r):
        r.done = self.clock()
        self.used -= r.n * STATE_BYTES_PER_PARTICLE
        if not self.keep_results:
            r.cell = r.off = r.u = None
        self.finished.append(r)

    def _reap(self, block: bool = False) -> int:
        """Complete the rounds whose events have passed (block: wait for the
        oldest one at least).  Returns how many rounds were completed."""
        done = 0
        while self.inflight:
            ev, slot, plan = self.inflight[0]
            if not ev.query():
                if not (block and done == 0):
                    break
                ev.synchronize()
            self.inflight.pop(0)
            done += 1
            for r, s in plan:
                r.remaining -= s
                self.psteps += r.n * s
                if r.remaining == 0:
                    self.active.remove(r)
                    self._finish(r)
        if not self.inflight and self._busy_from is not None:
            self.busy_s += self.clock() - self._busy_from
            self._busy_from = None
        return done

    def round(self) -> bool:
        """Complete finished rounds, admit, and enqueue one round if any
        admitted request has steps left to schedule (waiting for a work list
        only when both are in flight).  Returns True if a round was enqueued."""
        self._reap()
        self._admit()
        todo = [r for r in self.active if r.unplanned > 0]
        if not todo:
            return False
        if len(self.inflight) >= self.PIPELINE:   # both work lists in use
            self._reap(block=True)
        slot = self._slot
        self._slot = (self._slot + 1) % self.PIPELINE
        its = self.item_arrays[slot]
        steps = self._steps_this_round(todo)
        # costliest items first: the kernel's CTAs claim items in list order,
        # so the round ends evenly (longest-processing-time-first)
        todo.sort(key=lambda r: -steps[id(r)])
        k = 0
        plan = []
        for r in todo:
            s = steps[id(r)]
            nchunks = (r.n + self.chunk - 1) // self.chunk
            if k + nchunks > self.max_items:
                break
            blk = its[k:k + nchunks]
            first = np.arange(nchunks, dtype=np.int64) * self.chunk
            blk["cell"] = r.cell.data_ptr()
            blk["off"] = r.off.data_ptr()
            blk["u"] = r.u.data_ptr()
            blk["stride"] = r.n
            blk["first"] = first
            blk["count"] = np.minimum(self.chunk, r.n - first)
            blk["nsteps"] = s
            blk["snapshot"] = r.snapshot
            blk["reserved"] = 0
            blk["q_over_m"] = r.q_over_m
            blk["dt"] = r.dt
            k += nchunks
            r.unplanned -= s
            plan.append((r, s))
        if self._busy_from is None:
            self._busy_from = self.clock()
        self._check(self.L.part_server_run(self.hs[slot], k))
        ev = self.torch.cuda.Event()
        ev.record(self.stream)
        self.inflight.append((ev, slot, plan))
        self.rounds += 1
        return True

    def _steps_this_round(self, todo):
        """Steps each request advances in this round (see round_psteps)."""
        if not self.round_psteps:
            return {id(r): min(r.unplanned, self.slice_steps) for r in todo}
        budget = float(self.round_psteps)
        out, rest = {}, list(todo)
        while rest:      # water-filling: whole remainders that fit an equal share
            share = budget / len(rest)
            fits = [r for r in rest if r.n * r.unplanned <= share]
            if not fits:
                break
            for r in fits:
                out[id(r)] = r.unplanned
                budget -= r.n * r.unplanned
            rest = [r for r in rest if id(r) not in out]
        for r in rest:
            out[id(r)] = min(r.unplanned, int(budget / len(rest) / r.n))
        # never fewer than slice_steps: large requests keep their pace
        for r in todo:
            out[id(r)] = max(out[id(r)], min(r.unplanned, self.slice_steps))
        return out

    def drain(self):
        """Wait for every enqueued round and complete its requests."""
        while self.inflight:
            self._reap(block=True)
        for h in self.hs:
            self._check(self.L.part_server_sync(h))

    def run_until_idle(self):
        while self.queue or self.active or self.inflight:
            if not self.round():
                if self.inflight:
                    self._reap(block=True)
                elif self.queue:
                    raise RuntimeError("queued request cannot be admitted")
        self.drain()

    def stats(self):
        lat = np.array([r.latency for r in self.finished if r.latency is not None])
        return {"completed": len(self.finished), "rounds": self.rounds,
                "particle_steps": int(self.psteps),
                "busy_s": self.busy_s,
                "throughput_busy": self.psteps / self.busy_s if self.busy_s else None,
                "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_s": float(np.percentile(lat, 99)) if lat.size else None}


# ---------------------------------------------------------------------- autotuner
def autotune(torch, snapshots, candidates=None, n=1 << 21, slices=4, cache_path=None):
    """Pick the serving shape by timing a fixed synthetic batch per candidate:
    (threads per CTA, persistent CTAs per SM, chunk = particles per work item,
    i.e. the tile of sorted cells one CTA takes at a time, slice = steps per
    round).  One thread advances one particle.  Each candidate runs n
    particles for `slices` rounds after a warm-up round; the result is cached
    in a JSON file keyed by device name and snapshot grids."""
    cache_path = cache_path or os.environ.get(
        "PART_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache",
                                            "paper_2602_23434_b300_autotune.json"))
    candidates = candidates or [(t, c, ch, sl) for (t, c) in ((256, 4), (512, 4), (256, 8))
                                for ch in (2048, 8192) for sl in (16, 64)]
    key = json.dumps([torch.cuda.get_device_name(), [s.n_cells for s in snapshots], n, slices,
                      [list(c) for c in candidates]])
    try:
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return cache[key]
    except (OSError, ValueError):  # no cache yet, or an unreadable one
        cache = {}
    best, results = None, []
    for t, c, ch, sl in candidates:
        srv = Server(torch, snapshots, mem_budget_bytes=n * STATE_BYTES_PER_PARTICLE * 2,
                     chunk=ch, slice_steps=sl, threads=t, ctas_per_sm=c)
        srv.submit(len(snapshots) - 1, n, sl * (slices + 1), seed=7)
        srv.round()                                   # warm-up round (admits, captures)
        srv.drain()
        t0 = time.perf_counter()
        while srv.active or srv.inflight:
            srv.round()
        srv.drain()
        el = time.perf_counter() - t0
        rate = n * sl * slices / el
        results.append({"threads": t, "ctas_per_sm": c, "chunk": ch, "slice_steps": sl,
                        "psteps_per_s": rate})
        if best is None or rate > best["psteps_per_s"]:
            best = results[-1]
        srv.close()
    out = dict(best)
    out["candidates"] = results
    cache[key] = out
    try:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f)
    except OSError:  # a read-only location only costs the next run a re-tune
        pass
    return out
