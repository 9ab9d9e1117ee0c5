"""Continuous-batching server for isolated-system solves.

Requests (cubic mesh N, dtype, arrival time) are admitted in arrival order
while a stream slot is free and the device memory they need fits the budget;
admitted solves run concurrently on the slots' streams, and each completion
frees its slot and memory for the next admission.  Latency is completion time
minus arrival time.

Memory accounting (the admission budget):
* plans are pooled by (N, dtype) and reused; a plan's workspace counts while
  the plan exists, idle or busy; idle plans are destroyed least recently used
  first when an admission needs room;
* every cached Green's spectrum counts (the library keeps one per doubled
  mesh and dtype);
* each in-flight request counts its output buffer.

Plan creation (the Green's spectrum on a cache miss, the y-pass timing) can
run off the admission path (``async_plans=True``): a request whose (N, dtype)
has no idle plan reserves the plan's bytes and has it built on a background
thread, and stays queued while requests behind it whose plans are ready are
admitted (within a look-ahead window).  Its latency then includes the plan's
creation: misses are served cold, not hidden by a warm-up.

Size-aware admission (``express_slots``): the last few slots take only
cheap requests (estimated device time at most ``express_cost``, see
``request_cost``), so a burst of large solves cannot hold every slot while
small requests queue behind it; large requests keep their arrival order on
the other slots.

The device side is behind a small backend interface (``TorchBackend`` here;
tests substitute a fake one), so the admission and pooling logic is plain
host code.
"""
import collections
import concurrent.futures as cf
import math
import threading
import time

import numpy as np

from . import native, sources

OK = "ok"


class Request:
    __slots__ = ("id", "n", "dtype", "seed", "arrival", "admitted", "finished", "status", "slot", "plan", "out",
                 "handle")

    def __init__(self, rid, n, dtype, seed=0, arrival=0.0):
        self.id = rid
        self.n = int(n)
        self.dtype = dtype
        self.seed = seed
        self.arrival = float(arrival)
        self.admitted = None
        self.finished = None
        self.status = None
        self.slot = None
        self.plan = None
        self.out = None
        self.handle = None

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


# device time of a solve relative to FP32 at the same N: FP64 runs on the
# FP64 units (25.8x FP32 at 256^3), float pairs on the FP32 units (5.4x)
DTYPE_COST = {"f32": 1.0, "df64": 5.4, "f64": 25.8}


def request_cost(n, dtype):
    """Relative device time of one solve of a cubic mesh of n cells."""
    return DTYPE_COST.get(dtype, 1.0) * float(n) ** 3


class PlanPool:
    """Plans keyed by (N, dtype); a plan serves one request at a time."""

    def __init__(self, backend):
        self.backend = backend
        self.idle = collections.OrderedDict()  # plan id -> (key, plan), LRU order
        self.workspace = {}                    # plan id -> bytes
        self.bytes = 0

    def take_idle(self, key):
        for pid, (k, plan) in self.idle.items():
            if k == key:
                del self.idle[pid]
                return plan
        return None

    def evict_one(self):
        if not self.idle:
            return False
        pid, (k, plan) = self.idle.popitem(last=False)
        self.bytes -= self.workspace.pop(pid)
        self.backend.destroy_plan(plan)
        return True

    def add(self, plan, nbytes):
        self.workspace[id(plan)] = nbytes
        self.bytes += nbytes

    def release(self, key, plan):
        self.idle[id(plan)] = (key, plan)

    def close(self):
        while self.evict_one():
            pass


class Server:
    """Admission by memory budget over `slots` concurrent streams.

    on_finish: called with each completed request before its output is
    dropped (unless keep_outputs), e.g. to check or copy it.
    async_plans: create missing plans on background threads (`plan_workers`
    of them); admission then looks at up to `lookahead` queued requests for
    one whose plan is ready.
    express_slots: slots kept for requests of request_cost <= express_cost
    (default: an FP32 solve of 128^3); such requests take an express slot
    first, then any slot; admission then also looks past large requests
    that wait for a slot (which keep their order among themselves).
    """

    def __init__(self, backend, budget_bytes=120e9, slots=8, keep_outputs=False, on_finish=None,
                 async_plans=False, lookahead=64, express_slots=0, express_cost=None, plan_workers=1):
        self.backend = backend
        self.budget = float(budget_bytes)
        self.slots = int(slots)
        self.keep_outputs = keep_outputs
        self.on_finish = on_finish
        self.pool = PlanPool(backend)
        self.inflight_bytes = 0
        self.peak_bytes = 0
        self.async_plans = async_plans
        if not 0 <= int(express_slots) < int(slots):
            raise ValueError("express_slots must leave at least one slot for every request")
        self.express_slots = int(express_slots)
        self.express_cost = request_cost(128, "f32") if express_cost is None else float(express_cost)
        self.lookahead = int(lookahead) if (async_plans or self.express_slots) else 1
        self.pending = {}          # key -> (future, reserved bytes)
        self.pending_bytes = 0
        # background plan creation: `plan_workers` threads (the backend gives
        # each its own set-up stream)
        self.factory = cf.ThreadPoolExecutor(max_workers=max(1, int(plan_workers))) if async_plans else None

    def small(self, req):
        return self.express_slots > 0 and request_cost(req.n, req.dtype) <= self.express_cost

    def _pick_slot(self, free, small):
        """A free slot for a request: small ones take an express slot first,
        large ones only the others; None if there is none."""
        if not self.express_slots:
            return free[-1]
        first_express = self.slots - self.express_slots
        normal = [s for s in free if s < first_express]
        if small:
            express = [s for s in free if s >= first_express]
            return (express or normal)[-1]
        return normal[-1] if normal else None

    def used(self):
        return self.pool.bytes + self.backend.spectrum_bytes() + self.inflight_bytes + self.pending_bytes

    def _collect_plans(self):
        """Move finished background plan creations into the pool."""
        for key, (fut, reserved) in list(self.pending.items()):
            if not fut.done():
                continue
            del self.pending[key]
            self.pending_bytes -= reserved
            try:
                plan, nbytes = fut.result()
            except native.IsofftError as e:
                self.failed[key] = e.status
                continue
            self.pool.add(plan, nbytes)
            self.pool.release(key, plan)

    def _admit(self, req, slot):
        key = (req.n, req.dtype)
        out_bytes = self.backend.output_bytes(req.n, req.dtype)
        if key in self.failed:
            req.status = "error:%d" % self.failed.pop(key)
            return "reject"
        plan = self.pool.take_idle(key)
        if plan is None:
            if key in self.pending:
                return "pending"
            need = self.backend.plan_bytes(req.n, req.dtype) + out_bytes
            if need > self.budget:
                req.status = "budget_exceeded"
                return "reject"
            while self.used() + need > self.budget:
                if not self.pool.evict_one():
                    return "wait"
            if self.async_plans:
                reserved = need - out_bytes
                self.pending[key] = (self.factory.submit(self.backend.create_plan, req.n, req.dtype), reserved)
                self.pending_bytes += reserved
                self.peak_bytes = max(self.peak_bytes, self.used())
                return "pending"
            try:
                plan, nbytes = self.backend.create_plan(req.n, req.dtype)
            except native.IsofftError as e:
                if e.status == native.IPF_OUT_OF_MEMORY and self.pool.evict_one():
                    return "wait"
                req.status = "error:%d" % e.status
                return "reject"
            self.pool.add(plan, nbytes)
        else:
            # room for the output: other idle plans go first (the one taken
            # is not idle, so it stays)
            while self.used() + out_bytes > self.budget:
                if not self.pool.evict_one():
                    self.pool.release(key, plan)
                    return "wait"
        req.plan = plan
        req.slot = slot
        req.out = self.backend.alloc_output(req.n, req.dtype)
        self.inflight_bytes += out_bytes
        req.handle = self.backend.submit(plan, req, slot)
        self.peak_bytes = max(self.peak_bytes, self.used())
        return "ok"

    def _finish(self, req, now):
        req.finished = now
        req.status = OK
        self.inflight_bytes -= self.backend.output_bytes(req.n, req.dtype)
        self.pool.release((req.n, req.dtype), req.plan)
        self.backend.retire(req)
        if self.on_finish is not None:
            self.on_finish(req)
        if not self.keep_outputs:
            req.out = None

    def run(self, requests, clock=None, idle_sleep=0.0):
        """Serve `requests` (sorted by arrival, seconds from the start) to
        completion; returns them with admitted/finished times and status."""
        clock = clock or time.perf_counter
        reqs = sorted(requests, key=lambda r: r.arrival)
        queue = []
        free = list(range(self.slots))
        inflight = {}
        self.failed = {}
        i = 0
        done = 0
        t0 = clock()
        while done < len(reqs):
            now = clock() - t0
            progressed = False
            while i < len(reqs) and reqs[i].arrival <= now:
                queue.append(reqs[i])
                i += 1
            for slot, req in list(inflight.items()):
                if self.backend.is_done(req):
                    self._finish(req, clock() - t0)
                    del inflight[slot]
                    free.append(slot)
                    done += 1
                    progressed = True
            if self.pending:
                self._collect_plans()
            # admission: the first `lookahead` queued requests in arrival
            # order; one waiting for memory stops the scan (nothing behind
            # it may take the memory it waits for), one whose plan is being
            # built is passed over, and so is a large request with no slot
            # of its kind free (and every large request behind it)
            j = 0
            large_blocked = False
            while j < len(queue) and j < self.lookahead and free:
                req = queue[j]
                small = self.small(req)
                slot = None if (large_blocked and not small) else self._pick_slot(free, small)
                if slot is None:
                    large_blocked = True
                    j += 1
                    continue
                verdict = self._admit(req, slot)
                if verdict == "wait" and not inflight and not self.pending:
                    # nothing will complete to make room: drop the cached
                    # spectra no plan references, then try once more
                    self.backend.trim_spectra()
                    verdict = self._admit(req, slot)
                    if verdict == "wait":
                        req.status = "budget_exceeded"
                        verdict = "reject"
                if verdict == "wait":
                    break
                if verdict == "pending":
                    j += 1
                    continue
                queue.pop(j)
                if verdict == "reject":
                    req.finished = clock() - t0
                    done += 1
                else:
                    req.admitted = clock() - t0
                    free.remove(slot)
                    inflight[slot] = req
                progressed = True
            if not progressed:
                if not inflight and not queue and not self.pending and i < len(reqs):
                    self.backend.wait_until(reqs[i].arrival + t0, clock)
                elif idle_sleep:
                    time.sleep(idle_sleep)
        return reqs

    def close(self):
        if self.factory is not None:
            for fut, _ in self.pending.values():
                try:
                    plan, _ = fut.result()
                    self.backend.destroy_plan(plan)
                except native.IsofftError:
                    pass
            self.pending.clear()
            self.pending_bytes = 0
            self.factory.shutdown(wait=True)
            self.factory = None
        self.pool.close()


def poisson_arrivals(count, rate, seed=0):
    """Arrival times of a Poisson process of `rate` requests per second."""
    g = sources.rng(seed)
    return np.cumsum(g.exponential(1.0 / rate, count))


def latency_stats(reqs):
    lat = np.array([r.latency for r in reqs if r.status == OK])
    if lat.size == 0:
        return {"count": 0}
    span = max(r.finished for r in reqs if r.status == OK) - min(r.arrival for r in reqs)
    return {"count": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "solves_per_s": float(lat.size / span) if span > 0 else None}


class TorchBackend:
    """The device side of the server: library plans, one torch stream per
    slot, a completion event per request, and a bank of client sources (one
    seeded multi-sphere source per (N, dtype), made before serving starts)."""

    def __init__(self, slots, device=0, express_slots=0):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        # the express slots (the last ones) run on high-priority streams: the
        # block scheduler gives their pending blocks the SMs that free up
        # before those of the other streams' queued kernels
        self.slots = slots
        self.set_express(express_slots)
        self._tls = threading.local()  # one set-up stream per plan-creating thread
        self.bank = {}

    def set_express(self, express_slots):
        """Give the last `express_slots` slots high-priority streams (the
        others normal ones)."""
        torch = self.torch
        self.streams = [torch.cuda.Stream(device=self.dev, priority=-1 if s >= self.slots - express_slots else 0)
                        for s in range(self.slots)]

    @property
    def setup_stream(self):
        st = getattr(self._tls, "stream", None)
        if st is None:
            st = self._tls.stream = self.torch.cuda.Stream(device=self.dev)
        return st

    def source(self, n, dtype):
        key = (n, dtype)
        if key not in self.bank:
            bodies = sources.multi_sphere_bodies(sources.rng(1000 + n))
            self.bank[key] = sources.rasterize_torch(bodies, (n, n, n), (1.0 / n,) * 3, device=self.dev,
                                                     dtype=self.torch.float32 if dtype == "f32"
                                                     else self.torch.float64)
        return self.bank[key]

    def prepare(self, requests):
        for r in requests:
            self.source(r.n, r.dtype)
        self.torch.cuda.synchronize(self.dev)

    def warm_spectra(self, requests):
        """Build the cached spectrum of every doubled mesh the requests use
        (the paper builds it once at initialisation)."""
        seen = set()
        for r in requests:
            key = (r.n, r.dtype)
            if key in seen:
                continue
            seen.add(key)
            p = native.ipf_plan_create((r.n,) * 3, (1.0 / r.n,) * 3, r.dtype, 0, 0, self.setup_stream.cuda_stream)
            native.ipf_plan_destroy(p)

    def plan_bytes(self, n, dtype):
        return native.ipf_estimate_bytes((n,) * 3, (1.0 / n,) * 3, dtype)

    def output_bytes(self, n, dtype):
        return n ** 3 * (4 if dtype == "f32" else 8)

    def spectrum_bytes(self):
        return native.ipf_greens_cache_bytes()

    def trim_spectra(self):
        native.ipf_greens_cache_trim(0)

    def create_plan(self, n, dtype):
        p = native.ipf_plan_create((n,) * 3, (1.0 / n,) * 3, dtype, 0, 0, self.setup_stream.cuda_stream)
        return p, native.ipf_plan_workspace_bytes(p)

    def destroy_plan(self, plan):
        native.ipf_plan_destroy(plan)

    def alloc_output(self, n, dtype):
        return self.torch.empty((n, n, n), dtype=self.torch.float32 if dtype == "f32" else self.torch.float64,
                                device=self.dev)

    def submit(self, plan, req, slot):
        st = self.streams[slot]
        src = self.source(req.n, req.dtype)
        req.out.record_stream(st)
        native.ipf_solve(plan, src.data_ptr(), req.out.data_ptr(), st.cuda_stream)
        ev = self.torch.cuda.Event()
        ev.record(st)
        return ev

    def is_done(self, req):
        return req.handle.query()

    def retire(self, req):
        req.handle = None

    def wait_until(self, t_abs, clock):
        while clock() < t_abs:
            pass


def saturated_throughput(server, backend, requests):
    """All requests arrive at once: the served solves per second."""
    reqs = [Request(r.id, r.n, r.dtype, r.seed, 0.0) for r in requests]
    server.run(reqs)
    return latency_stats(reqs)
