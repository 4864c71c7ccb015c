"""Continuous-batching serving loop for per-page morphology pipelines.

A request names a page that is already resident on the device and asks for
a pipeline of operations whose result is returned as a run-length image.
The default pipeline is close(31x1) -> open(3x3) -> dilate(1x15) -> RLE.

:class:`Server` runs an arrival schedule (e.g. Poisson) against an executor:

* requests that have arrived wait in a FIFO queue;
* a request is admitted when a slot (pre-allocated device buffers: the
  intermediate pages, the RLE output, its batch workspace) is free and its
  bytes fit the memory budget beside everything in flight;
* every loop iteration launches ONE persistent batch for all requests
  admitted since the last launch, on the next stream of a small pool, while
  earlier batches may still be running — requests that arrive while others
  are on the GPU are admitted as slots free up and their work overlaps on
  the device (continuous batching, not a queue alone);
* completions are detected by CUDA events; a request's latency runs from its
  arrival to the completion of its batch.

:class:`PerPageExecutor` is the unbatched baseline: one request at a time, each
operation its own launch on one stream, synchronised before the next request.

The scheduling logic (queue, admission, slots, statistics) is plain Python
and runs with any executor, which is how the CPU tests exercise it with a
fake one.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

DEFAULT_PIPELINE = (("close", (31, 1)), ("open", (3, 3)), ("dilate", (1, 15)))


def poisson_arrivals(rate: float, n: int, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of n requests of a Poisson process."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def percentiles(lat_ms):
    if len(lat_ms) == 0:
        return {"p50_ms": None, "p99_ms": None, "mean_ms": None, "max_ms": None}
    a = np.asarray(lat_ms)
    return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
            "mean_ms": float(a.mean()), "max_ms": float(a.max())}


@dataclass
class Request:
    rid: int
    page: int             # index into the server's page pool
    arrival: float        # seconds since the start of the run
    admitted: float = -1.0
    done: float = -1.0
    slot: int = -1


@dataclass
class Stats:
    completed: int = 0
    latencies_ms: list = field(default_factory=list)
    queue_ms: list = field(default_factory=list)
    max_in_flight: int = 0
    max_in_flight_bytes: int = 0
    launches: int = 0
    batch_sizes: list = field(default_factory=list)
    wall_s: float = 0.0

    def summary(self):
        d = percentiles(self.latencies_ms)
        d.update({"completed": self.completed, "launches": self.launches,
                  "mean_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
                  "max_in_flight": self.max_in_flight,
                  "max_in_flight_bytes": self.max_in_flight_bytes,
                  "sustained_pages_s": self.completed / self.wall_s if self.wall_s > 0 else 0.0,
                  "queue_p99_ms": percentiles(self.queue_ms)["p99_ms"]})
        return d


class Server:
    """Admission, slots and the launch / completion loop (executor-agnostic).

    executor: object with ``slot_bytes`` (bytes one request holds while in
    flight), ``n_slots``, ``launch(requests) -> handle``, ``done(handle) ->
    bool`` and ``release(handle)``.
    """

    def __init__(self, executor, budget_bytes: float = 40e9, clock=time.perf_counter,
                 idle_sleep: float = 20e-6):
        self.ex = executor
        self.budget = float(budget_bytes)
        self.clock = clock
        self.idle_sleep = idle_sleep
        max_by_budget = int(self.budget // max(1, executor.slot_bytes))
        if max_by_budget < 1:
            raise ValueError("one request (%d bytes) does not fit the budget" % executor.slot_bytes)
        self.n_slots = min(executor.n_slots, max_by_budget)

    def run(self, arrivals, pages, time_limit: float = None) -> Stats:
        reqs = [Request(i, int(p), float(t)) for i, (t, p) in enumerate(zip(arrivals, pages))]
        pending = collections.deque()
        free = list(range(self.n_slots))[::-1]
        inflight = []          # (handle, [requests])
        st = Stats()
        nxt = 0
        in_flight_bytes = 0
        t0 = self.clock()
        while True:
            now = self.clock() - t0
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                pending.append(reqs[nxt])
                nxt += 1
            # admission: a free slot and room in the budget
            batch = []
            while pending and free and in_flight_bytes + self.ex.slot_bytes <= self.budget:
                r = pending.popleft()
                r.slot = free.pop()
                r.admitted = now
                in_flight_bytes += self.ex.slot_bytes
                batch.append(r)
            if batch:
                h = self.ex.launch(batch)
                inflight.append((h, batch))
                st.launches += 1
                st.batch_sizes.append(len(batch))
            n_in = sum(len(b) for _, b in inflight)
            st.max_in_flight = max(st.max_in_flight, n_in)
            st.max_in_flight_bytes = max(st.max_in_flight_bytes, in_flight_bytes)
            # completions
            still = []
            for h, b in inflight:
                if self.ex.done(h):
                    tdone = self.clock() - t0
                    for r in b:
                        r.done = tdone
                        st.latencies_ms.append(1e3 * (r.done - r.arrival))
                        st.queue_ms.append(1e3 * (r.admitted - r.arrival))
                        free.append(r.slot)
                        in_flight_bytes -= self.ex.slot_bytes
                        st.completed += 1
                    self.ex.release(h)
                else:
                    still.append((h, b))
            inflight = still
            if nxt >= len(reqs) and not pending and not inflight:
                break
            if time_limit is not None and now > time_limit:
                break
            if not inflight and not pending and self.idle_sleep and nxt < len(reqs):
                # idle: sleep until shortly before the next arrival, then spin
                gap = reqs[nxt].arrival - (self.clock() - t0) - 2e-4
                if gap > 0:
                    time.sleep(min(gap, 1e-3))
        st.wall_s = (self.clock() - t0) - (reqs[0].arrival if reqs else 0.0)
        self.requests = reqs
        return st


# ------------------------------------------------------------ executors

class _Slots:
    """Pre-allocated device buffers of every slot."""

    def __init__(self, M, torch, W, H, n_slots, n_ops, runs_per_row, device):
        nw = (W + 63) // 64
        self.mid = [[M.Packed(torch.empty((H, nw), dtype=torch.int64, device=device), W)
                     for _ in range(n_ops)] for _ in range(n_slots)]
        cap = H * min(runs_per_row, (W + 1) // 2)
        self.out = [M.Rle.empty(W, H, cap, device=device) for _ in range(n_slots)]
        self.page_bytes = H * nw * 8
        self.cap = cap


class BatchExecutor:
    """Continuous batching: one persistent batch launch per admission round,
    on a pool of streams; each request's pipeline is chained jobs (the job
    of step k depends on step k-1), ending with a bitmap->RLE job.

    Host cost per launch is kept small: the job descriptors of every
    (slot, page) pair are built once; a round with one request reuses a plan
    already on the device (launch = one memset + one kernel); a larger round
    concatenates the cached descriptors, builds its plan in C into a pinned
    staging buffer and uploads it asynchronously on the round's stream."""

    def __init__(self, pool, W, H, n_slots=64, pipeline=DEFAULT_PIPELINE, n_streams=4,
                 runs_per_row=None, path="packed", device="cuda"):
        import ctypes
        import torch
        from . import morph as M
        self.ct, self.M, self.torch = ctypes, M, torch
        self.lib = M.lib()
        self.pool = pool                      # list of Packed pages on the device
        self.pipeline = pipeline
        self.path = path
        self.W, self.H = W, H
        self.device = device
        rpr = runs_per_row if runs_per_row else W // 8 + 4
        self.slots = _Slots(M, torch, W, H, n_slots, len(pipeline), rpr, device)
        self.n_slots = n_slots
        self.jpr = len(pipeline) + 1          # jobs per request
        self.streams = [torch.cuda.Stream(device=device) for _ in range(n_streams)]
        self.k = 0
        self._desc = {}                       # (slot, page) -> morph_job array of one request
        self._plans = {}                      # (slot, page) -> (dev plan, host plan)
        # sizes of the largest round (every slot in one launch)
        big = self._array([(s, 0) for s in range(n_slots)])
        self.max_plan = int(self.lib.morph_batch_plan_bytes(big, n_slots * self.jpr, 0, 0))
        host = np.zeros(self.max_plan, np.uint8)
        M._check(self.lib.morph_batch_plan_build(host.ctypes.data, self.max_plan, big,
                                                 n_slots * self.jpr, 0, 0))
        self.max_ws = int(self.lib.morph_batch_workspace_size(host.ctypes.data))
        self.ws = [torch.empty(self.max_ws, dtype=torch.uint8, device=device) for _ in self.streams]
        self.staging = [torch.empty(self.max_plan, dtype=torch.uint8, pin_memory=True)
                        for _ in self.streams]
        self.dplan = [torch.empty(self.max_plan, dtype=torch.uint8, device=device) for _ in self.streams]
        self.staged = [None] * len(self.streams)
        self.slot_bytes = (len(pipeline) * self.slots.page_bytes + self.slots.cap * 4 + 4 * (H + 1)
                           + self.max_ws // n_slots)

    def _request_desc(self, slot, page):
        key = (slot, page)
        arr = self._desc.get(key)
        if arr is None:
            M = self.M
            arr = (M.morph_job * self.jpr)()
            src = self.pool[page]
            for k, (op, (sw, sh)) in enumerate(self.pipeline):
                j = arr[k]
                j.op, j.path = M.OPS[op], (M.PATH_RLE if self.path == "rle" else M.PATH_PACKED)
                j.se_w, j.se_h, j.origin_x, j.origin_y = sw, sh, sw // 2, sh // 2
                j.depends_on = k - 1
                j.src = src.desc()
                dst = self.slots.mid[slot][k]
                j.dst = dst.desc()
                src = dst
            j = arr[self.jpr - 1]
            j.op, j.depends_on = M.TO_RLE, self.jpr - 2
            j.se_w = j.se_h = 1
            j.src = src.desc()
            j.dst = self.slots.out[slot].desc()
            self._desc[key] = arr
        return arr

    def _array(self, pairs):
        ct = self.ct
        n = len(pairs) * self.jpr
        arr = (self.M.morph_job * n)()
        size = ct.sizeof(self.M.morph_job) * self.jpr
        for i, (slot, page) in enumerate(pairs):
            ct.memmove(ct.addressof(arr) + i * size, self._request_desc(slot, page), size)
            for k in range(self.jpr):
                if arr[i * self.jpr + k].depends_on >= 0:
                    arr[i * self.jpr + k].depends_on += i * self.jpr
        return arr

    def launch(self, reqs):
        torch, lib = self.torch, self.lib
        si = self.k % len(self.streams)
        self.k += 1
        stream = self.streams[si]
        h = stream.cuda_stream
        if len(reqs) == 1:
            key = (reqs[0].slot, reqs[0].page)
            plan = self._plans.get(key)
            if plan is None:
                arr = self._request_desc(*key)
                nb = int(lib.morph_batch_plan_bytes(arr, self.jpr, 0, 0))
                host = np.zeros(nb, np.uint8)
                self.M._check(lib.morph_batch_plan_build(host.ctypes.data, nb, arr, self.jpr, 0, 0))
                plan = (torch.from_numpy(host).to(self.device), host)
                self._plans[key] = plan
            dev, host = plan
            self.M._check(lib.morph_batch_launch(dev.data_ptr(), host.ctypes.data,
                                                 self.ws[si].data_ptr(), self.max_ws, 0, h))
        else:
            arr = self._array([(r.slot, r.page) for r in reqs])
            n = len(reqs) * self.jpr
            if self.staged[si] is not None:
                self.staged[si].synchronize()   # the previous upload from this buffer is done
            stg = self.staging[si]
            nb = int(lib.morph_batch_plan_bytes(arr, n, 0, 0))
            self.M._check(lib.morph_batch_plan_build(stg.data_ptr(), nb, arr, n, 0, 0))
            with torch.cuda.stream(stream):
                self.dplan[si][:nb].copy_(stg[:nb], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(stream)
            self.staged[si] = ev
            self.M._check(lib.morph_batch_launch(self.dplan[si].data_ptr(), stg.data_ptr(),
                                                 self.ws[si].data_ptr(), self.max_ws, 0, h))
        ev = torch.cuda.Event()
        ev.record(stream)
        return ev

    def done(self, h):
        return h.query()

    def release(self, h):
        pass

    def result(self, r):
        return self.slots.out[r.slot]


class PerPageExecutor:
    """Unbatched baseline: each operation is its own launch on one stream and
    the request is synchronised before the next one is started."""

    def __init__(self, pool, W, H, pipeline=DEFAULT_PIPELINE, runs_per_row=None, device="cuda"):
        import torch
        from . import morph as M
        self.M, self.torch = M, torch
        self.pool = pool
        self.pipeline = pipeline
        rpr = runs_per_row if runs_per_row else W // 8 + 4
        self.slots = _Slots(M, torch, W, H, 1, len(pipeline), rpr, device)
        self.n_slots = 1
        self.slot_bytes = len(pipeline) * self.slots.page_bytes + self.slots.cap * 4
        self.ws = torch.empty(M.convert_workspace_size(H), dtype=torch.uint8, device=device)

    def launch(self, reqs):
        for r in reqs:
            src = self.pool[r.page]
            for k, (op, (sw, sh)) in enumerate(self.pipeline):
                dst = self.slots.mid[0][k]
                self.M.morph_rect(op, dst, src, sw, sh)
                src = dst
            self.M.rle_from_bitmap(self.slots.out[0], src, self.ws)
        self.torch.cuda.synchronize()
        return None

    def done(self, h):
        return True

    def release(self, h):
        pass
