"""Continuous-batching server for test-particle tracing requests.

Requests (N particles, S Boris steps, one of several field snapshots that stay
resident on the device) arrive at any time.  Each scheduling round:
  1. admits queued requests in arrival order while their particle state fits
     in the device-memory budget (admission by free HBM), initialises them on
     the device (Philox draws, then a cell sort for gather locality);
  2. cuts every active request into work items of `chunk` particles that
     advance min(remaining, slice_steps) steps;
  3. runs the round through the C ABI (one persistent kernel replayed from a
     CUDA graph), waits for it, and completes the requests that are done.
Requests that arrive while others are on the GPU join at the next round, so
their work overlaps on the device with the running ones.  All arithmetic runs
in libpart.so; this module schedules and bookkeeps only.
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
    remaining: int = 0
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
    def __init__(self, torch, snapshots, mem_budget_bytes: int, max_items: int = 1 << 16,
                 chunk: int = 2048, slice_steps: int = 32, threads: int = 256,
                 ctas_per_sm: int = 4, clock=time.perf_counter):
        self.torch = torch
        self.L = P.lib()
        self.snaps = snapshots
        self.stream = snapshots[0].part.stream
        self.budget = int(mem_budget_bytes)
        self.chunk = int(chunk)
        self.slice_steps = int(slice_steps)
        self.max_items = int(max_items)
        self.clock = clock
        dbytes, hbytes = C.c_size_t(), C.c_size_t()
        self._check(self.L.part_server_sizes(len(snapshots), max_items, C.byref(dbytes),
                                             C.byref(hbytes)))
        dev = snapshots[0].part.device
        self.ws = torch.empty(dbytes.value, dtype=torch.uint8, device=dev)
        self.stage = torch.empty(hbytes.value, dtype=torch.uint8, pin_memory=True)
        arr = (C.c_void_p * len(snapshots))(*[s.part.ctx.value for s in snapshots])
        self.h = C.c_void_p()
        self._check(self.L.part_server_init(C.byref(self.h), arr, len(snapshots), max_items,
                                            C.c_void_p(self.ws.data_ptr()), dbytes.value,
                                            C.c_void_p(self.stage.data_ptr()), hbytes.value,
                                            C.c_void_p(self.stream.cuda_stream), threads,
                                            ctas_per_sm))
        self.items = self.L.part_server_items(self.h)
        self.queue: list[Request] = []
        self.active: list[Request] = []
        self.finished: list[Request] = []
        self.used = 0
        self.rounds = 0
        self.busy_s = 0.0
        self.psteps = 0
        self._next = 0

    def _check(self, code):
        if code != 0:
            msg = self.L.part_last_error(None)
            raise P.PartError(code, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.part_server_sync(self.h)
            self.L.part_server_destroy(self.h)
            self.h = C.c_void_p()

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
        r.remaining = int(steps)
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
            sp.sync()                      # sorted state into the request's arrays
            self.used += need
            r.admitted = self.clock()
            if r.remaining == 0:
                self._finish(r)
            else:
                self.active.append(r)

    def _finish(self, r):
        r.done = self.clock()
        self.used -= r.n * STATE_BYTES_PER_PARTICLE
        self.finished.append(r)

    def round(self) -> bool:
        """One scheduling round; returns False when there was nothing to run."""
        self._admit()
        if not self.active:
            return False
        its = self.items
        k = 0
        plan = []
        for r in self.active:
            s = min(r.remaining, self.slice_steps)
            nchunks = (r.n + self.chunk - 1) // self.chunk
            if k + nchunks > self.max_items:
                break
            for c in range(nchunks):
                w = its[k]
                w.cell, w.off, w.u = r.cell.data_ptr(), r.off.data_ptr(), r.u.data_ptr()
                w.stride = r.n
                w.first = c * self.chunk
                w.count = min(self.chunk, r.n - c * self.chunk)
                w.nsteps = s
                w.snapshot = r.snapshot
                w.reserved = 0
                w.q_over_m = r.q_over_m
                w.dt = r.dt
                k += 1
            plan.append((r, s))
        t0 = self.clock()
        self._check(self.L.part_server_run(self.h, k))
        self._check(self.L.part_server_sync(self.h))
        self.busy_s += self.clock() - t0
        self.rounds += 1
        still = []
        planned = {id(r) for r, _ in plan}
        for r, s in plan:
            r.remaining -= s
            self.psteps += r.n * s
        for r in self.active:
            if id(r) in planned and r.remaining == 0:
                self._finish(r)
            else:
                still.append(r)
        self.active = still
        return True

    def run_until_idle(self):
        while self.queue or self.active:
            if not self.round() and self.queue:
                raise RuntimeError("queued request cannot be admitted")

    def stats(self):
        lat = np.array([r.latency for r in self.finished if r.latency is not None])
        return {"completed": len(self.finished), "rounds": self.rounds,
                "particle_steps": int(self.psteps),
                "busy_s": self.busy_s,
                "throughput_busy": self.psteps / self.busy_s if self.busy_s else None,
                "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_s": float(np.percentile(lat, 99)) if lat.size else None}


# ---------------------------------------------------------------------- autotuner
def autotune(torch, snapshots, candidates=None, n=1 << 21, steps=16, cache_path=None):
    """Pick (threads, ctas_per_sm, chunk) of the serving kernel by timing one
    round of a fixed synthetic batch per candidate; cached in a JSON file
    keyed by device name and snapshot grids."""
    cache_path = cache_path or os.environ.get(
        "PART_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache",
                                            "paper_2602_23434_b300_autotune.json"))
    key = json.dumps([torch.cuda.get_device_name(), [s.n_cells for s in snapshots], n, steps])
    try:
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return cache[key]
    except (OSError, ValueError):  # no cache yet, or an unreadable one
        cache = {}
    candidates = candidates or [(t, c, ch) for t in (128, 256, 512) for c in (2, 4, 8)
                                for ch in (1024, 4096)]
    best, results = None, []
    for t, c, ch in candidates:
        srv = Server(torch, snapshots, mem_budget_bytes=n * STATE_BYTES_PER_PARTICLE * 2,
                     chunk=ch, slice_steps=steps, threads=t, ctas_per_sm=c)
        r = srv.submit(len(snapshots) - 1, n, steps * 3, seed=7)
        srv.round()                                   # warm-up round (also admits)
        t0 = time.perf_counter()
        srv.round()
        srv.round()
        el = time.perf_counter() - t0
        rate = 2 * n * steps / el
        results.append({"threads": t, "ctas_per_sm": c, "chunk": ch, "psteps_per_s": rate})
        if best is None or rate > best["psteps_per_s"]:
            best = results[-1]
        srv.close()
        del r
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
