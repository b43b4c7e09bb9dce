"""Serving loop: channel solves arriving over time, run to steady state with
continuous batching on the multi-solve engine.

Requests (velocity set, Hermite order, Nx, Ny, Kn, tolerance on max|du|) are
admitted into engine slots as soon as a slot and arena memory are free
(admission by HBM footprint, first fit over the queue so one large request
does not block smaller ones); all resident solves advance together one chunk
at a time; after every chunk each solve whose last step changed u_x by less
than its tolerance is harvested (mass flow, slip velocity) and its memory
freed for the queue.  Requests that arrive while others are running join at
the next chunk boundary.

Precision routing: the loop can drive several engines at once (each on its
own stream, so their chunks overlap on the GPU) and send each request to one
of them.  ``PrecisionRouter`` sends a request to fp64 storage when its
stopping decision is at risk in fp32: the per-step change of u_x that the
tolerance test compares is only known to ~2e-10 from fp32 populations, and a
test that lands on the other side of the tolerance stops the solve one chunk
earlier or later, which moves the reported mass flow by ~chunk x tol / u.

``serve_plain`` is the comparison path: the same requests solved one at a
time with the single-solve fp64 API.
"""
import math
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    t_arrival: float
    dvm: str
    order: int
    Nx: int
    Ny: int
    Kn: float
    tol: float
    mach: float = 1e-3
    # filled in by the server
    t_admit: float = math.nan
    t_done: float = math.nan
    steps: int = 0
    mdot: float = math.nan
    us: float = math.nan
    du: float = math.nan
    converged: bool = False
    status: int = 0
    lane: str = ""

    @property
    def force(self):
        """g = 8 tau Ma (no-slip Navier-Stokes centre speed Ma c0), tau = sqrt(2/pi) Kn."""
        return 8.0 * math.sqrt(2.0 / math.pi) * self.Kn * self.mach

    @property
    def latency(self):
        return self.t_done - self.t_arrival


def requests_from_workload(items):
    return [Request(i, it["t_arrival"], it["dvm"], it["order"], it["Nx"], it["Ny"], it["Kn"],
                    it["tol"]) for i, it in enumerate(items)]


@dataclass
class ServeStats:
    completed: int
    wall_s: float
    solves_per_s: float
    p50_s: float
    p99_s: float
    mean_queue_s: float
    max_resident: int
    chunks: int
    cell_steps: float
    extra: dict = field(default_factory=dict)

    def as_dict(self):
        d = {k: getattr(self, k) for k in ("completed", "wall_s", "solves_per_s", "p50_s", "p99_s",
                                          "mean_queue_s", "max_resident", "chunks", "cell_steps")}
        d.update(self.extra)
        return d


def _stats(done, t0, t1, max_resident, chunks, cell_steps):
    ok = [r for r in done if r.status == 0]
    lat = np.array([r.latency for r in ok]) if ok else np.array([math.nan])
    q = np.array([r.t_admit - r.t_arrival for r in ok]) if ok else np.array([math.nan])
    wall = max(t1 - t0, 1e-9)
    st = ServeStats(len(ok), wall, len(ok) / wall, float(np.percentile(lat, 50)),
                    float(np.percentile(lat, 99)), float(np.mean(q)), max_resident, chunks,
                    cell_steps)
    st.extra["failed"] = len(done) - len(ok)
    return st


def relaxation_steps(r, c):
    """Time constant, in steps, of the slowest (viscous) mode of a channel
    request: l0^2 / (pi^2 nu) with nu = tau = sqrt(2/pi) Kn (Eq. nm.11, nm.13)
    and dt = 1 / (Ny c), i.e. Ny c / (pi^2 tau)."""
    tau = math.sqrt(2.0 / math.pi) * r.Kn
    return r.Ny * c / (math.pi ** 2 * tau)


class PrecisionRouter:
    """Send a request to fp64 storage when fp32 may flip its stopping chunk.

    Near the stop the per-step change du decays by exp(-chunk / T) per
    chunk (T = relaxation_steps); fp32 populations know du only to about
    `du_noise` (measured ~2e-10 at Ma 1e-3), and the maximum over the nodes
    of |du + noise| is biased upward by a few times that, so the test
    du < tol lands on the wrong side of a chunk boundary with probability
    about (du_noise / tol) x T / chunk.  Requests above `risk` go to "fp64",
    the others to "fp32".  The default 1e-4 is the largest threshold at
    which no fp32-served request of the 60 s config-5 stream (12,000
    requests) missed the fp64 result by more than 1e-4 in mass flow."""

    def __init__(self, velocity_sets, chunk=100, du_noise=2e-10, risk=1e-4):
        self.c = {name: float(v[2]) for name, v in velocity_sets.items()}
        self.chunk, self.du_noise, self.risk = chunk, du_noise, risk

    def flip_risk(self, r):
        return self.du_noise / r.tol * relaxation_steps(r, self.c[r.dvm]) / self.chunk

    def __call__(self, r):
        return "fp64" if self.flip_risk(r) > self.risk else "fp32"


class _Lane:
    """One engine of the batcher with its resident solves and in-flight chunks."""

    def __init__(self, engine):
        self.engine = engine
        self.active = {}                   # slot -> Request
        self.inflight = []                 # snapshots of launched, unharvested chunks
        self.chunks = 0


class ContinuousBatcher:
    """Drive one engine (paper_1510_08886_gb300.Engine, or any object with
    add/remove/run/chunk, and optionally launch/wait), or several engines
    keyed by name with `route(request) -> name`, with a request queue."""

    def __init__(self, engine, velocity_sets, max_steps=200000, clock=time.perf_counter,
                 route=None):
        engines = engine if isinstance(engine, dict) else {"main": engine}
        self.lanes = {k: _Lane(e) for k, e in engines.items()}
        self.route = route if route is not None else (lambda r: next(iter(self.lanes)))
        self.sets = velocity_sets          # name -> (e, w, c)
        self.max_steps = max_steps
        self.clock = clock
        self.queue = []
        self.done = []
        self.cell_steps = 0.0
        self.max_resident = 0

    # single-engine views (the common case)
    @property
    def engine(self):
        return next(iter(self.lanes.values())).engine

    @property
    def active(self):
        out = {}
        for lane in self.lanes.values():
            out.update(lane.active)
        return out if len(self.lanes) > 1 else next(iter(self.lanes.values())).active

    @property
    def chunks(self):
        return sum(l.chunks for l in self.lanes.values())

    def _busy(self):
        return any(l.active or l.inflight for l in self.lanes.values())

    def submit(self, req):
        self.queue.append(req)

    def admit(self):
        """First fit over the queue in arrival order, each request into its
        routed engine.  A request the engine rejects (unknown velocity set,
        invalid arguments) is answered at once with its error code instead of
        stopping the server."""
        still = []
        full = set()
        for i, r in enumerate(self.queue):
            if len(full) == len(self.lanes):
                still.extend(self.queue[i:])      # every engine's slots taken: the rest waits
                break
            try:
                name = self.route(r)
                lane = self.lanes[name]
            except KeyError as err:
                r.status = getattr(err, "code", -1)
                r.t_admit = r.t_done = self.clock()
                self.done.append(r)
                continue
            cap = getattr(lane.engine, "max_solves", None)
            if cap is not None and len(lane.active) >= cap:
                full.add(name)
                still.append(r)                   # no free slot in that engine: waits
                continue
            try:
                e, w, c = self.sets[r.dvm]
                slot = lane.engine.add(e, w, c, r.order, r.Nx, r.Ny, r.Kn, r.force)
            except (KeyError, ValueError, RuntimeError) as err:
                r.status = getattr(err, "code", -1)
                r.t_admit = r.t_done = self.clock()
                self.done.append(r)
                continue
            if slot is None:
                still.append(r)
                continue
            r.t_admit = self.clock()
            r.lane = name
            lane.active[slot] = r
        self.queue = still
        self.max_resident = max(self.max_resident,
                                sum(len(l.active) for l in self.lanes.values()))

    def _launch_snapshot(self, lane):
        """Count one chunk for every resident solve of a lane; return (slot,
        request, steps after the chunk) for the harvest of that chunk."""
        lane.chunks += 1
        K = lane.engine.chunk
        self.cell_steps += sum(r.Nx * r.Ny for r in lane.active.values()) * K
        snap = []
        for slot, r in lane.active.items():
            r.steps += K
            snap.append((slot, r, r.steps))
        return snap

    def _harvest(self, lane, res, snap):
        """Retire the solves of a finished chunk whose result meets their
        tolerance, ran out of steps or turned non-finite (du NaN or inf)."""
        live = [(s, r, st) for s, r, st in snap if lane.active.get(s) is r]
        if not live:
            return 0
        now = self.clock()
        slots = np.array([s for s, _, _ in live], dtype=np.int64)
        du = res[slots, 0]
        tol = np.array([r.tol for _, r, _ in live])
        steps = np.array([st for _, _, st in live])
        done = ~(np.isfinite(du) & (du >= tol)) | (steps >= self.max_steps)
        finished = []
        for i in np.nonzero(done)[0]:
            slot, r, d = int(slots[i]), live[i][1], float(du[i])
            status = 0 if math.isfinite(d) else -5
            r.status, r.du, r.steps = status, d, int(steps[i])
            r.converged = status == 0 and d < r.tol
            r.mdot, r.us = float(res[slot, 1]), float(res[slot, 2])
            r.t_done = now
            finished.append(slot)
        for slot in finished:
            lane.engine.remove(slot)
            self.done.append(lane.active.pop(slot))
        return len(finished)

    def step(self):
        """Admit, advance every resident solve by one chunk, harvest.

        With engines that can launch asynchronously (launch/wait), every
        lane's next chunk is queued before the previous one's results are
        processed, so the GPU runs while the host harvests and admits: a
        solve is harvested from the results of the chunk that met its
        tolerance (its reported steps are that chunk's), it has already
        been queued for one more chunk by then, and an admitted request
        joins one chunk later."""
        self.admit()
        n = 0
        for lane in self.lanes.values():
            if not hasattr(lane.engine, "launch"):
                if lane.active:
                    res = lane.engine.run(1)
                    n += self._harvest(lane, res, self._launch_snapshot(lane))
                continue
            if lane.active:
                lane.engine.launch(1)
                lane.inflight.append(self._launch_snapshot(lane))
        for lane in self.lanes.values():
            if not hasattr(lane.engine, "launch"):
                continue
            if lane.inflight and (len(lane.inflight) == 2 or not lane.active):
                res = lane.engine.wait()
                n += self._harvest(lane, res, lane.inflight.pop(0))
        return n

    def serve(self, requests, realtime=True, time_limit=None):
        """Play a request stream (t_arrival relative to the start) and return
        ServeStats.  With realtime=False, arrival times are ignored (every
        request is queued at once)."""
        pending = sorted(requests, key=lambda r: r.t_arrival)
        t0 = self.clock()
        i = 0
        while i < len(pending) or self.queue or self._busy():
            now = self.clock()
            if time_limit is not None and now - t0 > time_limit:
                break
            while i < len(pending) and (not realtime or pending[i].t_arrival <= now - t0):
                r = pending[i]
                r.t_arrival = t0 + r.t_arrival if realtime else t0
                self.submit(r)
                i += 1
            if not self.queue and not self._busy() and i < len(pending):
                time.sleep(max(0.0, min(0.01, pending[i].t_arrival - (self.clock() - t0))))
                continue
            self.step()
        return _stats(self.done, t0, self.clock(), self.max_resident, self.chunks, self.cell_steps)


def serve_plain(requests, make_solver, realtime=True, time_limit=None, check_every=100,
                max_steps=200000, clock=time.perf_counter):
    """Comparison path: requests solved one at a time in arrival order with
    the single-solve API (make_solver(request) -> Solver with run_to_steady).
    Requests still waiting when time_limit expires are not counted."""
    pending = sorted(requests, key=lambda r: r.t_arrival)
    t0 = clock()
    done = []
    cell_steps = 0.0
    for r in pending:
        now = clock()
        if time_limit is not None and now - t0 > time_limit:
            break
        arrival = t0 + r.t_arrival if realtime else t0
        if realtime and arrival > now:
            time.sleep(arrival - now)
        r.t_arrival = arrival
        r.t_admit = clock()
        s = make_solver(r)
        conv, steps, du = s.run_to_steady(r.tol, max_steps, check_every)
        r.converged, r.steps, r.du = conv, steps, du
        r.mdot, r.us = s.mass_flow(), s.slip_velocity()
        r.t_done = clock()
        cell_steps += r.Nx * r.Ny * steps
        done.append(r)
    return _stats(done, t0, clock(), 1, 0, cell_steps)
