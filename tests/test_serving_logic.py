"""Host logic of the continuous-batching server, on CPU with a fake device
backend (simulated clock and solve durations): the memory budget is never
exceeded, admission is first-come first-served, plans are reused, oversize
requests and failed plan creations are rejected without stalling the rest."""
import numpy as np
import pytest

from paper_1106_0557_gb300 import native, serving


class FakeClock:
    def __init__(self, dt=1e-5):
        self.t = 0.0
        self.dt = dt

    def __call__(self):
        self.t += self.dt
        return self.t


class FakeBackend:
    def __init__(self, clock, fail=(), spectrum=1000):
        self.clock = clock
        self.fail = set(fail)
        self.created = 0
        self.destroyed = 0
        self.live = set()
        self.spectra = spectrum

    def plan_bytes(self, n, dtype):
        return 2 * n ** 3 * (8 if dtype == "f32" else 16)

    def output_bytes(self, n, dtype):
        return n ** 3 * (4 if dtype == "f32" else 8)

    def spectrum_bytes(self):
        return self.spectra

    def trim_spectra(self):
        self.spectra = 0

    def create_plan(self, n, dtype):
        if (n, dtype) in self.fail:
            raise native.IsofftError(native.IPF_OUT_OF_MEMORY, "create")
        self.created += 1
        p = object()
        self.live.add(id(p))
        return p, self.plan_bytes(n, dtype)

    def destroy_plan(self, plan):
        self.destroyed += 1
        self.live.discard(id(plan))

    def alloc_output(self, n, dtype):
        return np.zeros(1)

    def submit(self, plan, req, slot):
        return self.clock.t + 1e-4 * (req.n / 16.0) ** 3 * (8 if req.dtype == "f64" else 1)

    def is_done(self, req):
        return self.clock.t >= req.handle

    def retire(self, req):
        pass

    def wait_until(self, t_abs, clock):
        self.clock.t = max(self.clock.t, t_abs)


def make_requests(count, seed=0, lo=8, hi=48, rate=None):
    g = np.random.default_rng(seed)
    arr = serving.poisson_arrivals(count, rate, seed) if rate else np.zeros(count)
    return [serving.Request(i, int(g.integers(lo, hi)), "f32" if g.uniform() < 0.7 else "f64", i, arr[i])
            for i in range(count)]


def test_budget_respected_and_all_complete():
    clock = FakeClock()
    be = FakeBackend(clock)
    budget = 3 * FakeBackend(clock).plan_bytes(48, "f64")
    srv = serving.Server(be, budget_bytes=budget, slots=4)
    reqs = srv.run(make_requests(300, rate=2000.0), clock=clock)
    assert all(r.status == serving.OK for r in reqs)
    assert srv.peak_bytes <= budget
    srv.close()
    assert be.live == set()


def test_first_come_first_served():
    clock = FakeClock()
    srv = serving.Server(FakeBackend(clock), budget_bytes=1e12, slots=3)
    reqs = srv.run(make_requests(100, seed=3, rate=500.0), clock=clock)
    adm = [r.admitted for r in sorted(reqs, key=lambda r: r.arrival)]
    assert adm == sorted(adm)
    assert all(r.admitted >= r.arrival for r in reqs)
    assert all(r.finished > r.admitted for r in reqs)


def test_plans_are_reused():
    clock = FakeClock()
    be = FakeBackend(clock)
    srv = serving.Server(be, budget_bytes=1e12, slots=2)
    reqs = [serving.Request(i, 32, "f32", i, 0.0) for i in range(50)]
    srv.run(reqs, clock=clock)
    assert be.created <= 2
    assert all(r.status == serving.OK for r in reqs)


def test_oversize_and_failed_requests_do_not_stall_the_rest():
    clock = FakeClock()
    be = FakeBackend(clock, fail={(40, "f64")})
    budget = be.plan_bytes(64, "f32") + be.output_bytes(64, "f32") + be.spectrum_bytes()
    srv = serving.Server(be, budget_bytes=budget, slots=2)
    reqs = [serving.Request(0, 16, "f32", 0, 0.0), serving.Request(1, 200, "f32", 1, 0.0),
            serving.Request(2, 40, "f64", 2, 0.0), serving.Request(3, 24, "f32", 3, 0.0)]
    srv.run(reqs, clock=clock)
    st = {r.id: r.status for r in reqs}
    assert st[0] == serving.OK and st[3] == serving.OK
    assert st[1] == "budget_exceeded"
    assert st[2] == "error:%d" % native.IPF_OUT_OF_MEMORY
    assert srv.peak_bytes <= budget


def test_spectra_trimmed_when_nothing_in_flight():
    clock = FakeClock()
    be = FakeBackend(clock, spectrum=10 ** 9)
    need = be.plan_bytes(32, "f32") + be.output_bytes(32, "f32")
    srv = serving.Server(be, budget_bytes=need + 10, slots=1)
    reqs = srv.run([serving.Request(0, 32, "f32", 0, 0.0)], clock=clock)
    assert reqs[0].status == serving.OK
    assert be.spectra == 0


def test_poisson_arrivals_and_stats():
    t = serving.poisson_arrivals(20000, rate=1000.0, seed=1)
    assert np.all(np.diff(t) >= 0)
    assert np.mean(np.diff(t)) == pytest.approx(1e-3, rel=0.05)
    clock = FakeClock()
    srv = serving.Server(FakeBackend(clock), budget_bytes=1e12, slots=4)
    reqs = srv.run(make_requests(200, seed=5, rate=3000.0), clock=clock)
    st = serving.latency_stats(reqs)
    assert st["count"] == 200 and 0 < st["p50_ms"] <= st["p99_ms"]


def test_async_plans_respect_budget_and_complete():
    """Plans built on the background thread: the budget (with the bytes
    reserved for plans being built) is never exceeded, every request
    completes, failed creations are rejected, and plans are reused."""
    clock = FakeClock()
    be = FakeBackend(clock, fail={(40, "f64")})
    budget = 3 * be.plan_bytes(48, "f64")
    srv = serving.Server(be, budget_bytes=budget, slots=4, async_plans=True, lookahead=16)
    reqs = make_requests(300, rate=2000.0)
    reqs.append(serving.Request(300, 40, "f64", 300, 0.05))
    srv.run(reqs, clock=clock)
    st = {r.id: r.status for r in reqs}
    assert st[300] == "error:%d" % native.IPF_OUT_OF_MEMORY
    assert all(s == serving.OK for i, s in st.items() if not (reqs[i].n == 40 and reqs[i].dtype == "f64"))
    assert srv.peak_bytes <= budget
    srv.close()
    assert be.live == set()
    # with room for every plan, each shape's plan is built once and reused
    clock = FakeClock()
    be = FakeBackend(clock)
    srv = serving.Server(be, budget_bytes=1e12, slots=4, async_plans=True)
    reqs = [serving.Request(i, 32 if i % 2 else 24, "f32", i, 0.0) for i in range(60)]
    srv.run(reqs, clock=clock)
    assert all(r.status == serving.OK for r in reqs)
    assert be.created <= 8
    srv.close()


def test_async_lookahead_passes_requests_waiting_for_a_plan():
    """A request whose plan is being built does not hold back a later request
    whose plan is ready; with look-ahead off (synchronous plans) admission is
    in arrival order."""
    clock = FakeClock()
    be = FakeBackend(clock)
    srv = serving.Server(be, budget_bytes=1e12, slots=2, async_plans=True, lookahead=8)
    srv.run([serving.Request(0, 16, "f32", 0, 0.0)], clock=clock)  # a ready plan of N = 16
    reqs = [serving.Request(1, 32, "f32", 1, 0.0), serving.Request(2, 16, "f32", 2, 0.0)]
    srv.run(reqs, clock=clock)
    assert all(r.status == serving.OK for r in reqs)
    assert reqs[1].admitted <= reqs[0].admitted
    srv.close()


def test_express_slot_serves_small_requests_past_a_burst_of_large_ones():
    """With one of four slots kept for cheap requests, small requests that
    arrive behind a burst of large ones run at once on that slot; the large
    ones never take it and keep their arrival order."""
    clock = FakeClock()
    be = FakeBackend(clock)
    srv = serving.Server(be, budget_bytes=1e12, slots=4, express_slots=1)
    big = [serving.Request(i, 48, "f64", i, 0.0) for i in range(8)]
    small = [serving.Request(100 + i, 16, "f32", i, 1e-4) for i in range(4)]
    assert not any(srv.small(r) for r in big) and all(srv.small(r) for r in small)
    srv.run(big + small, clock=clock)
    assert all(r.status == serving.OK for r in big + small)
    assert all(r.slot < 3 for r in big)
    assert max(r.finished for r in small) < max(r.admitted for r in big)
    adm = [r.admitted for r in big]
    assert adm == sorted(adm)
    # without the express slot the small requests wait for the large ones
    clock = FakeClock()
    srv = serving.Server(FakeBackend(clock), budget_bytes=1e12, slots=4)
    big = [serving.Request(i, 48, "f64", i, 0.0) for i in range(8)]
    small = [serving.Request(100 + i, 16, "f32", i, 1e-4) for i in range(4)]
    srv.run(big + small, clock=clock)
    assert min(r.admitted for r in small) > max(r.admitted for r in big)


def test_express_slots_keep_the_budget_and_complete_a_mix():
    clock = FakeClock()
    be = FakeBackend(clock, fail={(40, "f64")})
    budget = 3 * be.plan_bytes(48, "f64")
    srv = serving.Server(be, budget_bytes=budget, slots=4, express_slots=1, async_plans=True, lookahead=16,
                         express_cost=serving.request_cost(24, "f32"))
    reqs = make_requests(300, rate=2000.0)
    srv.run(reqs, clock=clock)
    st = [r.status for r in reqs]
    assert all(s == serving.OK or (r.n == 40 and r.dtype == "f64") for s, r in zip(st, reqs))
    assert srv.peak_bytes <= budget
    big = sorted((r for r in reqs if r.status == serving.OK and not srv.small(r)), key=lambda r: r.arrival)
    assert all(r.slot < 3 for r in big)
    srv.close()
    assert be.live == set()
    with pytest.raises(ValueError):
        serving.Server(be, slots=2, express_slots=2)
