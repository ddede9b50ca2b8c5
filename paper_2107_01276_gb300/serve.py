"""Serving loop: many independent adaptive simulations on one GPU.

Requests (a workload, a step count, an adaptation interval) arrive over
time.  The server admits a request when a slot is free and the device has
room for it (free HBM, from cudaMemGetInfo, minus a reserve), keeps its
particle state resident in its own library context on its own CUDA stream,
and advances it on a worker thread; the workers' kernels overlap on the
device.  As requests finish, their slots and memory go to waiting ones
(continuous batching).  The report gives per-step latency percentiles
beside the aggregate throughput.

With batch=True the requests step together instead, once set up on their
workers: a BatchStepper thread advances all of them in flight per tick,
first one sph_batch_adapt over those due for adaptation (their
adaptations in lockstep, one synchronisation per phase for all of them),
then one sph_batch_step over all (every per-particle phase of all of them
in one persistent launch), members joining as they are admitted and
leaving as they finish.  Requests with and without adaptation have a
stepper each, so a plain step never waits for an adaptation.

Every step of every simulation runs in the library's kernels (sph.py is the
binding); this module only schedules.  The ctypes calls release the GIL, so
the workers drive their contexts concurrently.
"""
from __future__ import annotations

import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import sph
from . import workloads as wl

# Device bytes one context holds per particle of capacity (state and its
# double buffer, pass outputs and records, sort scratch, cell table, anchor
# records, neighbour lists with 48 entries a particle, staging rows), with
# a margin; the background construction context counts the same per
# background slot.
BYTES_PER_SLOT = 1280


@dataclass
class Request:
    """One simulation: `workload` is a dict from workloads.py; it runs
    `steps` PEC steps with one sph_adapt call every `adapt_every` steps
    (0: none) after `refine` initial sph_adapt calls."""
    rid: int
    workload: dict
    steps: int
    adapt_every: int = 1
    refine: int = 0
    arrival: float = 0.0          # seconds after the start of the run
    precision: int = sph.SPH_MIXED
    capacity: int = 0             # 0: chosen from the workload
    bg_capacity: int = 0
    team: int = 0                 # pass A / B threads per particle (0: size rule)
    # filled in by the server
    admitted: float = float("nan")
    finished: float = float("nan")
    step_ms: list = field(default_factory=list)
    setup_s: float = 0.0          # admission to the first step
    background_s: float = 0.0     # of which: background construction
    particle_steps: int = 0
    final: dict | None = None
    error: str | None = None


def default_capacity(d: dict) -> int:
    n = len(d["particles"]["x"])
    return int(max(4 * n, 20000) if d.get("background") is not None else n + 16)


def estimate_bytes(req: Request) -> int:
    """Device memory the request's contexts will hold (upper estimate)."""
    d = req.workload
    cap = req.capacity or default_capacity(d)
    total = cap * BYTES_PER_SLOT
    if d.get("construct_background"):
        nb = len(d["background"]["x"])
        bcap = req.bg_capacity or max(100 * nb, 1 << 18)
        total += bcap * BYTES_PER_SLOT
    return int(total)


def _setup(req: Request, stream: int):
    """The request's context with its sets loaded, background built and
    initial refinement done."""
    d = req.workload
    cap = req.capacity or default_capacity(d)
    P = sph.make_params(d["params"], precision=req.precision, capacity=cap,
                        bg_capacity=req.bg_capacity)
    sim = sph.Simulation(P, stream)
    try:
        if req.team:
            sim.set_tuning(team_a=req.team, team_b=req.team)
        sim.load(d["particles"])
        if "walls" in d:
            sim.load(d["walls"], kind=sph.SPH_WALL)
        if "region" in d:
            sim.load(d["region"], kind=sph.SPH_REGION)
        if d.get("background") is not None:
            sim.load(d["background"], kind=sph.SPH_BACKGROUND)
            if d.get("construct_background"):
                t0 = time.perf_counter()
                sim.background()
                req.background_s = time.perf_counter() - t0
        for _ in range(req.refine):
            sim.adapt()
    except Exception:
        sim.close()
        raise
    return sim


def _finish(req: Request, sim, keep_final: bool):
    if keep_final:
        ids = sim.read("id")
        order = np.argsort(ids)
        req.final = {"id": ids[order]}
        for f in ("x", "y", "u", "v", "p", "m", "h"):
            req.final[f] = sim.read(f)[order]


def run_alone(req: Request, stream: int, keep_final: bool = True) -> Request:
    """Run one request to completion on `stream` (the worker body)."""
    t0 = time.perf_counter()
    sim = _setup(req, stream)
    req.setup_s = time.perf_counter() - t0
    try:
        for s in range(req.steps):
            t0 = time.perf_counter()
            if req.adapt_every and s % req.adapt_every == 0:
                sim.adapt()
            sim.step(1, want_time=True)          # synchronises: step done
            req.step_ms.append(1e3 * (time.perf_counter() - t0))
            req.particle_steps += sim.info()["n"]
        _finish(req, sim, keep_final)
    finally:
        sim.close()
    return req


class BatchStepper:
    """Continuous batching of the steps themselves: simulations join the
    ticks as they are admitted and leave when their steps are done.  A
    tick adapts the members due for adaptation (step s of a request with
    adapt_every > 0 and s % adapt_every == 0, as run_alone does) in one
    sph_batch_adapt, then steps every member in one sph_batch_step.  A
    step's latency is the tick's; a member whose adaptation fails leaves
    with its error while the others go on."""

    def __init__(self, max_instances: int, stream: int, batch=None):
        # batch: an object with adapt(sims, errors), step(sims, want_time),
        # set_graphs(bool) and close() (default: a library sph.Batch)
        self.batch = batch if batch is not None else sph.Batch(max_instances, stream)
        # members come and go, and the other workers allocate and
        # synchronise while a graph would be captured: launch by launch
        self.batch.set_graphs(False)
        self.cv = threading.Condition()
        self.members = []            # [sim, request, steps left, event, n, steps done]
        self.stop = False
        self.th = threading.Thread(target=self._loop, daemon=True)
        self.th.start()

    def advance(self, sim, req: Request):
        """Blocks until `sim` has made req.steps steps in the batch."""
        if req.steps <= 0:
            return
        ev = threading.Event()
        with self.cv:
            self.members.append([sim, req, req.steps, ev, sim.info()["n"], 0])
            self.cv.notify_all()
        ev.wait()
        if req.error:
            raise RuntimeError(req.error)

    def _loop(self):
        while True:
            with self.cv:
                while not self.members and not self.stop:
                    self.cv.wait()
                if not self.members:
                    return
                group = list(self.members)
            due = [m for m in group
                   if m[1].adapt_every and m[5] % m[1].adapt_every == 0]
            t0 = time.perf_counter()
            err = None
            bad = {}
            try:
                if due:
                    res = self.batch.adapt([m[0] for m in due], errors="return")
                    for m, r in zip(due, res):
                        if isinstance(r, tuple):
                            bad[id(m)] = "SphError: %s" % r[1]
                        else:
                            m[4] = r["n_after"]
                live = [m for m in group if id(m) not in bad]
                if live:
                    self.batch.step([m[0] for m in live], want_time=True)
            except Exception as e:            # every member fails
                err = "%s: %s" % (type(e).__name__, e)
            ms = 1e3 * (time.perf_counter() - t0)
            with self.cv:
                for m in group:
                    e = err or bad.get(id(m))
                    if e:
                        m[1].error = e
                        m[2] = 0
                    else:
                        m[1].step_ms.append(ms)
                        m[1].particle_steps += m[4]
                        m[2] -= 1
                        m[5] += 1
                    if m[2] <= 0:
                        self.members.remove(m)
                        m[3].set()

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        self.th.join()
        self.batch.close()


def run_batched(req: Request, stream: int, stepper: BatchStepper,
                keep_final: bool = True) -> Request:
    """A request set up on `stream`, then adapted and stepped by the batch
    stepper together with the others in flight."""
    t0 = time.perf_counter()
    sim = _setup(req, stream)
    req.setup_s = time.perf_counter() - t0
    try:
        stepper.advance(sim, req)
        _finish(req, sim, keep_final)
    finally:
        sim.close()
    return req


class Server:
    """Continuous-batching server.

    slots: requests in flight at most; reserve: bytes of free HBM never
    handed out; mem_info: callable returning (free, total) bytes (default
    torch.cuda.mem_get_info); runner: callable(request, stream) running one
    request (default run_alone); make_stream: callable returning a stream
    handle for a worker (default: a new torch CUDA stream); batch: the
    requests, once set up on their workers, adapt and step together
    through two BatchSteppers, one for the requests with adaptation and
    one for those without; make_stepper: callable(max_instances, stream)
    returning such a stepper (default BatchStepper), and batch_runner:
    callable(request, stream, stepper) running one request through it
    (default run_batched)."""

    def __init__(self, slots: int = 8, reserve: int = 2 << 30,
                 mem_info=None, runner=None, make_stream=None,
                 keep_final: bool = False, batch: bool = False,
                 make_stepper=None, batch_runner=None):
        self.slots = slots
        self.batch = batch
        self.make_stepper = make_stepper or BatchStepper
        self.batch_runner = batch_runner or \
            (lambda r, s, st: run_batched(r, s, st, self.keep_final))
        self.reserve = reserve
        self.keep_final = keep_final
        if mem_info is None:
            import torch
            mem_info = torch.cuda.mem_get_info
        self.mem_info = mem_info
        self.runner = runner or (lambda r, s: run_alone(r, s, self.keep_final))
        if make_stream is None:
            def make_stream():
                import torch
                st = torch.cuda.Stream()
                return st, st.cuda_stream
        self.make_stream = make_stream
        self._lock = threading.Lock()
        self._reserved = 0           # bytes promised to requests in flight
        self.admission_log = []      # (time, rid, "admit" | "wait" | "refuse")

    def _can_admit(self, req: Request) -> bool:
        free, _ = self.mem_info()
        need = estimate_bytes(req)
        return free - self._reserved - self.reserve >= need

    def run(self, requests, time_scale: float = 1.0) -> dict:
        """Serve `requests` (arrival times scaled by time_scale); returns
        the report."""
        pending = sorted(requests, key=lambda r: r.arrival)
        free_slots = list(range(self.slots))
        streams = [self.make_stream() for _ in range(self.slots)]
        threads = {}
        done = []
        cv = threading.Condition(self._lock)
        t_start = time.perf_counter()

        # two steppers: the requests with adaptation tick apart from those
        # without, so that a plain step never waits for an adaptation
        steppers = None
        if self.batch:
            steppers = {flag: self.make_stepper(self.slots, self.make_stream()[1])
                        for flag in (False, True)}

        def worker(slot, req):
            t0 = time.perf_counter()
            req.admitted = t0 - t_start
            try:
                if steppers is not None:
                    self.batch_runner(req, streams[slot][1],
                                      steppers[bool(req.adapt_every)])
                else:
                    self.runner(req, streams[slot][1])
            except Exception as e:            # reported, never fatal
                req.error = "%s: %s" % (type(e).__name__, e)
            req.finished = time.perf_counter() - t_start
            with cv:
                self._reserved -= estimate_bytes(req)
                free_slots.append(slot)
                done.append(req)
                cv.notify_all()

        with cv:
            while pending or len(done) < len(requests):
                now = time.perf_counter() - t_start
                admitted_any = False
                while pending and pending[0].arrival * time_scale <= now \
                        and free_slots:
                    req = pending[0]
                    if not self._can_admit(req):
                        if len(free_slots) == self.slots:
                            # nothing in flight will free memory: refuse
                            pending.pop(0)
                            req.error = "refused: needs %d bytes of device " \
                                "memory" % estimate_bytes(req)
                            req.admitted = req.finished = now
                            done.append(req)
                            self.admission_log.append((now, req.rid, "refuse"))
                            continue
                        self.admission_log.append((now, req.rid, "wait"))
                        break
                    pending.pop(0)
                    slot = free_slots.pop(0)
                    self._reserved += estimate_bytes(req)
                    self.admission_log.append((now, req.rid, "admit"))
                    th = threading.Thread(target=worker, args=(slot, req),
                                          daemon=True)
                    threads[req.rid] = th
                    th.start()
                    admitted_any = True
                if len(done) == len(requests):
                    break
                if not admitted_any:
                    wait = None
                    if pending and free_slots:
                        wait = max(0.0, pending[0].arrival * time_scale - now)
                        wait = min(wait, 0.05) if wait > 0 else 0.01
                    cv.wait(timeout=wait if wait is not None else 0.5)
        for th in threads.values():
            th.join()
        if steppers is not None:
            for st in steppers.values():
                st.close()
        wall = time.perf_counter() - t_start
        return self.report(requests, wall)

    @staticmethod
    def report(requests, wall: float) -> dict:
        lat = np.array([ms for r in requests for ms in r.step_ms]) \
            if any(r.step_ms for r in requests) else np.zeros(0)
        ps = sum(r.particle_steps for r in requests)
        return {
            "requests": len(requests),
            "failed": sum(1 for r in requests if r.error),
            "wall_s": wall,
            "particle_steps": ps,
            "particle_steps_per_s": ps / wall if wall > 0 else 0.0,
            "steps": int(lat.size),
            "step_ms_p50": float(np.percentile(lat, 50)) if lat.size else None,
            "step_ms_p99": float(np.percentile(lat, 99)) if lat.size else None,
            "queue_s_mean": float(np.mean([r.admitted - r.arrival for r in
                                           requests])) if requests else None,
            "setup_s_mean": float(np.mean([r.setup_s for r in requests]))
            if requests else None,
            "background_s_mean": float(np.mean([r.background_s for r in requests
                                                if r.background_s > 0]))
            if any(r.background_s > 0 for r in requests) else None,
            "step_s_total": float(sum(sum(r.step_ms) for r in requests) / 1e3),
            "errors": sorted({r.error for r in requests if r.error}),
        }


def c5_requests(n: int = 256, rate: float = 20.0, seed: int = 7,
                steps: int = 40, sizes=(5000, 200000)) -> list:
    """The serving workload's request stream: half flow past a cylinder
    (Re log-uniform in [20, 2000]), half Taylor-Green vortices (Re uniform
    in [50, 500]), particle counts log-uniform in `sizes`, Poisson arrivals
    at `rate` per second.  Cylinder sizes come from the finest spacing
    (D/ds_min between 25 and 100, about 3k to 30k fluid particles; the
    background construction grows as (D/ds_min)^2); Taylor-Green sizes from
    the lattice."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    lo, hi = math.log(sizes[0]), math.log(sizes[1])
    for k in range(n):
        t += rng.exponential(1.0 / rate)
        target = math.exp(rng.uniform(lo, hi))
        if k % 2 == 0:
            Re = math.exp(rng.uniform(math.log(20.0), math.log(2000.0)))
            # ~9k particles at D/50; the refined count grows ~ (D/ds_min)^1.2
            inv = min(100.0, max(25.0, 50.0 * (target / 9000.0) ** (1 / 1.2)))
            d = wl.cylinder(Re=Re, ds_min_over_D=1.0 / inv)
            bgc = int(1.5 * 101268 * (inv / 50.0) ** 2) + 50000
            # refined fluid: ~9k at D/50, growing about as (D/ds_min)^1.2
            cap = int(4 * 9000 * (inv / 50.0) ** 1.2) + 20000
            reqs.append(Request(k, d, steps, adapt_every=1, refine=12,
                                arrival=t, capacity=cap, bg_capacity=bgc))
        else:
            Re = rng.uniform(50.0, 500.0)
            nx = int(round(math.sqrt(target)))
            d = wl.taylor_green(nx=nx, Re=Re)
            reqs.append(Request(k, d, steps, adapt_every=0, arrival=t))
    return reqs
