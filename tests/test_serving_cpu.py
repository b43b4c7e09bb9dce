"""Host logic of the serving loop, with a fake engine on the CPU: admission by
footprint (first fit), continuous joining at chunk boundaries, harvesting
at each request's tolerance, statistics.  No GPU."""
import math

import numpy as np

from lbm_inputs import serving_workload
from paper_1510_08886_gb300.serving import (ContinuousBatcher, Request, requests_from_workload,
                                            serve_plain)


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeEngine:
    """Footprint = Nx*Ny bytes; du after n steps = 1e-3 exp(-n / (10 Ny Kn))."""

    def __init__(self, capacity, slots, chunk=100, clock=None, chunk_time=1e-3):
        self.capacity, self.chunk, self.clock, self.chunk_time = capacity, chunk, clock, chunk_time
        self.slots = [None] * slots
        self.results = np.zeros((slots, 4))
        self.peak_bytes = 0

    def used(self):
        return sum(s["bytes"] for s in self.slots if s)

    def add(self, e, w, c, order, Nx, Ny, Kn, force):
        need = Nx * Ny
        if self.used() + need > self.capacity:
            return None
        for i, s in enumerate(self.slots):
            if s is None:
                self.slots[i] = dict(bytes=need, steps=0, Ny=Ny, Kn=Kn, g=force)
                self.peak_bytes = max(self.peak_bytes, self.used())
                return i
        return None

    def remove(self, slot):
        assert self.slots[slot] is not None
        self.slots[slot] = None

    def run(self, chunks):
        for i, s in enumerate(self.slots):
            if s:
                s["steps"] += chunks * self.chunk
                T = 10.0 * s["Ny"] * s["Kn"]
                self.results[i] = [1e-3 * math.exp(-s["steps"] / T), 1.0 + s["Kn"], 0.5, 1e-3]
        if self.clock:
            self.clock.t += chunks * self.chunk_time
        return self.results

    def info(self, slot):
        return self.slots[slot]["steps"], 0


SETS = {"D2V16": (None, None, None)}


def _reqs(specs):
    return [Request(i, t, "D2V16", 3, 1, ny, kn, tol) for i, (t, ny, kn, tol) in enumerate(specs)]


def test_all_requests_complete_at_their_tolerance():
    clk = FakeClock()
    eng = FakeEngine(capacity=10_000, slots=8, clock=clk)
    b = ContinuousBatcher(eng, SETS, clock=clk)
    reqs = _reqs([(0.0, 64, 0.1, 1e-6), (0.0, 128, 0.5, 1e-8), (0.0, 32, 0.01, 1e-6)])
    st = b.serve(reqs, realtime=False)
    assert st.completed == 3
    for r in b.done:
        T = 10.0 * r.Ny * r.Kn
        assert r.converged and 1e-3 * math.exp(-r.steps / T) < r.tol
        # harvested at the first chunk boundary below tolerance
        assert 1e-3 * math.exp(-(r.steps - 100) / T) >= r.tol
        assert r.mdot == 1.0 + r.Kn


def test_admission_respects_footprint_and_first_fit():
    clk = FakeClock()
    eng = FakeEngine(capacity=1000, slots=16, clock=clk)
    b = ContinuousBatcher(eng, SETS, clock=clk)
    # a large request that must wait, then small ones that fit beside the first
    reqs = _reqs([(0.0, 600, 1.0, 1e-6), (0.0, 900, 1.0, 1e-6), (0.0, 100, 1.0, 1e-6),
                  (0.0, 200, 1.0, 1e-6)])
    b.serve(reqs, realtime=False)
    assert eng.peak_bytes <= 1000
    order = [r.rid for r in sorted(b.done, key=lambda r: r.t_admit)]
    assert order.index(2) < order.index(1)       # small request skipped the blocked large one
    assert all(r.converged for r in b.done)


def test_slots_limit_and_queue_wait():
    clk = FakeClock()
    eng = FakeEngine(capacity=10**9, slots=2, clock=clk)
    b = ContinuousBatcher(eng, SETS, clock=clk)
    reqs = _reqs([(0.0, 64, 0.1, 1e-6)] * 5)
    st = b.serve(reqs, realtime=False)
    assert st.completed == 5 and st.max_resident == 2
    waits = sorted(r.t_admit - r.t_arrival for r in b.done)
    assert waits[0] == 0.0 and waits[-1] > 0.0


def test_requests_join_at_chunk_boundaries_in_realtime():
    """Requests arriving while others run are admitted at the next chunk."""
    import time as _time

    eng = FakeEngine(capacity=10**9, slots=32, chunk=100, chunk_time=0.0)
    real_run = eng.run

    def slow_run(n):
        _time.sleep(0.002)
        return real_run(n)

    eng.run = slow_run
    b = ContinuousBatcher(eng, SETS)
    reqs = _reqs([(0.0, 400, 1.0, 1e-9), (0.02, 64, 0.1, 1e-6), (0.04, 64, 0.1, 1e-6)])
    st = b.serve(reqs, realtime=True)
    assert st.completed == 3
    first = next(r for r in b.done if r.rid == 0)
    later = [r for r in b.done if r.rid > 0]
    assert all(r.t_admit < first.t_done for r in later)   # joined while rid 0 was running
    assert st.max_resident >= 2


def test_stats_percentiles():
    clk = FakeClock()
    eng = FakeEngine(capacity=10**9, slots=64, clock=clk)
    b = ContinuousBatcher(eng, SETS, clock=clk)
    reqs = _reqs([(0.0, ny, 0.2, 1e-7) for ny in range(16, 80, 4)])
    st = b.serve(reqs, realtime=False)
    lat = np.array([r.latency for r in b.done])
    assert math.isclose(st.p50_s, np.percentile(lat, 50))
    assert math.isclose(st.p99_s, np.percentile(lat, 99))
    assert st.solves_per_s > 0 and st.cell_steps > 0


def test_serve_plain_sequential():
    class FakeSolver:
        def __init__(self, r):
            self.r = r

        def run_to_steady(self, tol, max_steps, check_every):
            return True, 500, tol / 2

        def mass_flow(self):
            return 2.0

        def slip_velocity(self):
            return 0.3

    reqs = _reqs([(0.0, 64, 0.1, 1e-6), (0.0, 64, 0.2, 1e-6)])
    st = serve_plain(reqs, FakeSolver, realtime=False)
    assert st.completed == 2 and all(r.steps == 500 and r.mdot == 2.0 for r in reqs)


def test_serving_workload_shape():
    items = serving_workload(duration_s=5.0)
    reqs = requests_from_workload(items)
    assert 700 < len(reqs) < 1300                      # Poisson, mean 200/s
    assert all(16 <= r.Ny <= 2048 and r.Nx == 1 and r.tol in (1e-6, 1e-8) for r in reqs)
    assert all(0.01 <= r.Kn <= 1.0 for r in reqs)
    gaps = np.diff([r.t_arrival for r in reqs])
    assert 0.003 < gaps.mean() < 0.007


def test_failures_do_not_stop_the_server():
    """A request with an unknown velocity set, one the engine rejects, and a
    solve whose state turns non-finite are answered with an error status while
    the other requests complete."""
    clk = FakeClock()

    class Faulty(FakeEngine):
        def add(self, e, w, c, order, Nx, Ny, Kn, force):
            if Ny == 13:
                err = RuntimeError("lbm_engine_add: invalid argument (-1)")
                err.code = -1
                raise err
            return super().add(e, w, c, order, Nx, Ny, Kn, force)

        def run(self, chunks):
            res = super().run(chunks)
            for i, s in enumerate(self.slots):
                if s and s["Ny"] == 17:
                    res[i, 0] = math.nan        # a NaN in the state makes du NaN
            return res

    eng = Faulty(capacity=10**9, slots=8, clock=clk)
    b = ContinuousBatcher(eng, SETS, clock=clk)
    reqs = _reqs([(0.0, 64, 0.1, 1e-6), (0.0, 13, 0.1, 1e-6), (0.0, 17, 0.1, 1e-6),
                  (0.0, 32, 0.2, 1e-6)])
    reqs.append(Request(4, 0.0, "NOPE", 3, 1, 32, 0.1, 1e-6))
    st = b.serve(reqs, realtime=False)
    by = {r.rid: r for r in b.done}
    assert by[0].converged and by[3].converged
    assert by[1].status == -1 and by[4].status == -1
    assert by[2].status == -5 and not by[2].converged
    assert st.completed == 2 and st.extra["failed"] == 3
    assert all(s is None for s in eng.slots)          # every slot released


def test_infinite_change_is_a_failure_and_full_slots_stop_admission():
    """A solve whose per-step change is infinite is answered as non-finite;
    with every slot taken, queued requests wait without being tried."""
    clk = FakeClock()

    class Inf(FakeEngine):
        max_solves = 2
        tries = 0

        def add(self, *a):
            Inf.tries += 1
            return super().add(*a)

        def run(self, chunks):
            res = super().run(chunks)
            for i, s in enumerate(self.slots):
                if s and s["Ny"] == 19:
                    res[i, 0] = math.inf
            return res

    eng = Inf(capacity=10**9, slots=2, clock=clk)
    b = ContinuousBatcher(eng, SETS, clock=clk)
    reqs = _reqs([(0.0, 19, 0.1, 1e-6), (0.0, 64, 0.1, 1e-6)] + [(0.0, 32, 0.1, 1e-6)] * 6)
    st = b.serve(reqs, realtime=False)
    by = {r.rid: r for r in b.done}
    assert by[0].status == -5 and not by[0].converged
    assert st.completed == 7 and st.extra["failed"] == 1
    assert Inf.tries == len(reqs)          # each request tried once: no retries while full


class PipeFake(FakeEngine):
    """FakeEngine with asynchronous chunks: a launch computes that chunk's
    results (the state after it), a wait hands them back oldest first."""

    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.q = []

    def launch(self, chunks):
        assert len(self.q) < 2
        self.q.append(self.run(chunks).copy())

    def wait(self):
        return self.q.pop(0)


def test_pipelined_chunks_give_the_same_answers():
    """Launching chunk k + 1 before harvesting chunk k: every request is
    answered from the chunk that met its tolerance, with the same step count
    and results as the synchronous loop (all requests admitted at once)."""
    specs = [(0.0, ny, kn, tol) for ny, kn, tol in
             [(64, 0.1, 1e-6), (128, 0.5, 1e-8), (32, 0.01, 1e-6), (200, 0.3, 1e-7),
              (16, 1.0, 1e-6), (90, 0.05, 1e-8)]]
    out = {}
    for cls in (FakeEngine, PipeFake):
        clk = FakeClock()
        eng = cls(capacity=10**9, slots=8, clock=clk)
        b = ContinuousBatcher(eng, SETS, clock=clk)
        st = b.serve(_reqs(specs), realtime=False)
        assert st.completed == len(specs)
        assert all(s is None for s in eng.slots)
        out[cls] = {r.rid: (r.steps, r.mdot, r.converged) for r in b.done}
    assert out[FakeEngine] == out[PipeFake]


def test_pipelined_slot_reuse_and_failures():
    """A slot freed by a harvest and taken by a new request while the next
    chunk (still holding the old solve) is in flight: the old solve's stale
    row is skipped; non-finite solves are answered with their status."""
    clk = FakeClock()

    class P(PipeFake):
        def run(self, chunks):
            res = super().run(chunks)
            for i, s in enumerate(self.slots):
                if s and s["Ny"] == 17:
                    res[i, 0] = math.nan
            return res

    eng = P(capacity=10**9, slots=2, clock=clk)
    b = ContinuousBatcher(eng, SETS, clock=clk)
    reqs = _reqs([(0.0, 16, 0.01, 1e-3), (0.0, 17, 0.1, 1e-6)] + [(0.0, 20 + i, 0.02, 1e-6)
                                                                    for i in range(5)])
    st = b.serve(reqs, realtime=False)
    by = {r.rid: r for r in b.done}
    assert by[1].status == -5
    assert st.completed == 6 and st.extra["failed"] == 1
    for r in b.done:
        if r.status == 0:
            T = 10.0 * r.Ny * r.Kn
            assert 1e-3 * math.exp(-r.steps / T) < r.tol          # converged at its steps
            assert 1e-3 * math.exp(-(r.steps - 100) / T) >= r.tol  # not a chunk earlier


def test_precision_router_risk_and_lanes():
    """Two engines behind one loop: the router's flip risk
    (du_noise / tol) x T / chunk with T = Ny c / (pi^2 tau) sends tight or
    slowly relaxing requests to "fp64"; each request is admitted, advanced
    and harvested in its own engine only, and every request completes."""
    from paper_1510_08886_gb300.serving import PrecisionRouter, relaxation_steps
    sets = {"D2V16": (None, None, 1.5)}
    router = PrecisionRouter(sets, chunk=100, du_noise=2e-10, risk=1e-3)
    assert PrecisionRouter(sets).risk == 1e-4
    r_fast = Request(0, 0.0, "D2V16", 3, 1, 16, 1.0, 1e-6)
    r_slow = Request(1, 0.0, "D2V16", 3, 1, 2000, 0.01, 1e-6)
    r_tight = Request(2, 0.0, "D2V16", 3, 1, 64, 0.1, 1e-8)
    tau = math.sqrt(2 / math.pi) * 0.01
    assert abs(relaxation_steps(r_slow, 1.5) - 2000 * 1.5 / (math.pi ** 2 * tau)) < 1e-9
    assert router(r_fast) == "fp32" and router(r_slow) == "fp64" and router(r_tight) == "fp64"
    assert abs(router.flip_risk(r_tight) / router.flip_risk(Request(3, 0.0, "D2V16", 3, 1, 64, 0.1,
                                                                    1e-6)) - 100) < 1e-9
    clk = FakeClock()
    engines = {"fp32": FakeEngine(10 ** 6, 8, clock=clk), "fp64": FakeEngine(10 ** 6, 8, clock=clk)}
    seen = {"fp32": set(), "fp64": set()}
    for name, eng in engines.items():
        orig = eng.add

        def add(*a, _orig=orig, _name=name):
            slot = _orig(*a)
            seen[_name].add((a[5], a[6]))     # (Ny, Kn)
            return slot
        eng.add = add
    reqs = [Request(i, 0.0, "D2V16", 3, 1, ny, kn, tol) for i, (ny, kn, tol) in
            enumerate([(16, 1.0, 1e-6), (2000, 0.01, 1e-6), (64, 0.1, 1e-8), (32, 0.5, 1e-6)] * 5)]
    b = ContinuousBatcher(engines, sets, clock=clk, route=router)
    st = b.serve(reqs, realtime=False)
    assert st.completed == len(reqs)
    assert all(r.lane == router(r) for r in reqs)
    assert seen["fp64"] == {(2000, 0.01), (64, 0.1)} and seen["fp32"] == {(16, 1.0), (32, 0.5)}
    assert all(r.converged for r in reqs)
