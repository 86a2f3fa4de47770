"""Host-side logic of the continuous-batching scheduler, driven by a fake
executor (no GPU): memory admission, slot limits, arrival order and latency
accounting."""
import pytest

from paper_2305_02064_gb300.serve import Arena, Scheduler, ServeRequest, latency_summary, poisson_arrivals


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3          # every look at the clock advances 1 ms
        return self.t


class FakeExecutor:
    """A request runs for `work` clock ticks after it starts."""

    def __init__(self, clock, work=5):
        self.clock, self.work = clock, work
        self.started, self.finished = [], []
        self.live = 0
        self.max_live = 0

    def start(self, req):
        self.started.append(req.rid)
        self.live += 1
        self.max_live = max(self.max_live, self.live)
        return {"req": req, "until": self.clock.t + self.work * 1e-3}

    def done(self, h):
        return self.clock.t >= h["until"]

    def finish(self, h):
        self.live -= 1
        self.finished.append(h["req"].rid)


def make(n, footprint, gap):
    return [ServeRequest(i, None, arrival=i * gap, footprint=footprint) for i in range(n)]


def test_memory_cap_limits_concurrency():
    clk = FakeClock()
    ex = FakeExecutor(clk, work=20)
    sch = Scheduler(ex, slots=8, mem_cap=100, clock=clk)
    done = sch.run(make(10, footprint=30, gap=0.0))
    assert len(done) == 10
    assert ex.max_live == 3                  # 3 x 30 <= 100 < 4 x 30
    assert sch.peak_in_use <= 100 and sch.in_use == 0


def test_slot_limit_and_fifo():
    clk = FakeClock()
    ex = FakeExecutor(clk, work=10)
    sch = Scheduler(ex, slots=2, mem_cap=10 ** 9, clock=clk)
    done = sch.run(make(6, footprint=1, gap=0.0))
    assert ex.max_live == 2
    assert ex.started == list(range(6))      # admitted in arrival order
    assert all(r.admitted >= r.arrival and r.completed > r.admitted for r in done)


def test_late_arrivals_join_running_work():
    """A request that arrives while others are running starts before they finish."""
    clk = FakeClock()
    ex = FakeExecutor(clk, work=50)
    sch = Scheduler(ex, slots=4, mem_cap=10 ** 9, clock=clk)
    reqs = make(3, footprint=1, gap=0.01)
    done = {r.rid: r for r in sch.run(reqs)}
    assert done[1].admitted < done[0].completed
    assert done[2].admitted < done[0].completed
    assert ex.max_live == 3


def test_oversized_request_is_rejected():
    clk = FakeClock()
    sch = Scheduler(FakeExecutor(clk), slots=2, mem_cap=10, clock=clk)
    with pytest.raises(ValueError):
        sch.run(make(1, footprint=11, gap=0.0))


def test_latency_summary_and_arrivals():
    clk = FakeClock()
    sch = Scheduler(FakeExecutor(clk, work=3), slots=1, mem_cap=10, clock=clk)
    done = sch.run(make(5, footprint=1, gap=0.0))
    s = latency_summary(done)
    assert s["n"] == 5 and s["p99_ms"] >= s["p50_ms"] > 0
    t = poisson_arrivals(2000, rate_hz=200.0, seed=1)
    assert (t[1:] > t[:-1]).all()
    assert 1 / 200 * 0.9 < (t[-1] / len(t)) < 1 / 200 * 1.1


def test_plan_cache_is_bounded_and_shares_plans(monkeypatch):
    """One plan per scan shape (plans are only read by the imaging calls),
    the least recently used evicted beyond the cache size."""
    import synth
    from paper_2305_02064_gb300 import batch
    monkeypatch.setattr(batch, "PLAN_CACHE_MAX", 3)
    batch._PLAN_CACHE.clear()
    scans = [synth.custom(nx_pos=2, ny_pos=2, nk=8, nx=8 + 8 * i, ny=8, nz=4) for i in range(5)]
    p0 = batch.plan_for(scans[0])
    assert batch.plan_for(scans[0]) is p0
    for s in scans[1:]:
        batch.plan_for(s)
    assert len(batch._PLAN_CACHE) == 3
    assert batch.plan_for(scans[0]) is not p0        # evicted, rebuilt
    batch._PLAN_CACHE.clear()


def test_arena_first_fit_all_or_nothing_and_merging():
    a = Arena(4096, align=256)
    p1 = a.place([100, 600])            # rounded to 256, 768
    assert p1 == [(0, 256), (256, 768)] and a.in_use == 1024
    p2 = a.place([2048])
    assert p2 == [(1024, 2048)]
    assert a.place([512, 1024]) is None  # 1024 left: the second block does not fit -> nothing placed
    assert a.in_use == 3072 and a.largest_free() == 1024
    a.release(p1)
    assert a.free == [(0, 1024), (3072, 1024)]
    a.release(p2)
    assert a.free == [(0, 4096)] and a.in_use == 0 and a.peak == 3072


class BlockExecutor(FakeExecutor):
    """A fake executor whose requests need device blocks of given sizes."""

    def __init__(self, clock, work, arena):
        super().__init__(clock, work)
        self.arena = arena

    def block_sizes(self, req):
        return req.scan


def test_scheduler_admits_by_arena_placement():
    """Requests wait until the arena can place all their blocks, whatever
    the footprints add up to; fragmentation is handled by first fit."""
    clk = FakeClock()
    arena = Arena(1000, align=1)
    ex = BlockExecutor(clk, work=20, arena=arena)
    reqs = [ServeRequest(i, [300, 100], arrival=0.0, footprint=0) for i in range(5)]
    sch = Scheduler(ex, slots=8, mem_cap=10 ** 9, clock=clk)
    done = sch.run(reqs)
    assert len(done) == 5 and ex.max_live == 2      # 2 x 400 <= 1000 < 3 x 400
    assert arena.peak <= 1000 and arena.in_use == 0 and arena.free == [(0, 1000)]
    with pytest.raises(ValueError):
        Scheduler(ex, slots=2, mem_cap=10 ** 9, clock=clk).run([ServeRequest(9, [600, 500], 0.0)])
