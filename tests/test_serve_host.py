"""Host logic of the serving loop (no GPU): admission by free device memory
and free slots, continuous batching as requests finish, refusal of a
request that can never fit, and the latency report."""
import threading
import time

from paper_2107_01276_gb300 import serve
from paper_2107_01276_gb300 import workloads as wl


class FakeDevice:
    """Free memory that shrinks while requests hold it."""

    def __init__(self, total):
        self.total = total
        self.used = 0
        self.lock = threading.Lock()
        self.peak_in_flight = 0
        self.in_flight = 0

    def mem_info(self):
        with self.lock:
            return self.total - self.used, self.total

    def runner(self, req, stream):
        need = serve.estimate_bytes(req)
        with self.lock:
            self.used += need
            self.in_flight += 1
            self.peak_in_flight = max(self.peak_in_flight, self.in_flight)
        for _ in range(req.steps):
            time.sleep(0.002)
            req.step_ms.append(2.0)
            req.particle_steps += 100
        with self.lock:
            self.used -= need
            self.in_flight -= 1


def _req(rid, nx, arrival, steps=5):
    return serve.Request(rid, wl.taylor_green(nx=nx), steps, adapt_every=0,
                         arrival=arrival)


def _server(dev, slots, reserve=0):
    return serve.Server(slots=slots, reserve=reserve, mem_info=dev.mem_info,
                        runner=dev.runner, make_stream=lambda: (None, 0))


def test_slots_bound_the_requests_in_flight():
    dev = FakeDevice(total=1 << 40)
    reqs = [_req(k, 20, 0.0) for k in range(7)]
    rep = _server(dev, slots=3).run(reqs)
    assert dev.peak_in_flight <= 3
    assert rep["requests"] == 7 and rep["failed"] == 0
    assert rep["steps"] == 35 and rep["particle_steps"] == 3500
    assert rep["step_ms_p50"] == 2.0 and rep["step_ms_p99"] == 2.0


def test_memory_bounds_admission_and_frees_on_completion():
    one = serve.estimate_bytes(_req(0, 30, 0.0))
    # room for two at a time (the server also counts its own promises)
    dev = FakeDevice(total=int(2.5 * one))
    reqs = [_req(k, 30, 0.0) for k in range(5)]
    srv = _server(dev, slots=8)
    rep = srv.run(reqs)
    assert rep["failed"] == 0
    assert dev.peak_in_flight == 1     # promise + holding: one fits at once
    kinds = [k for _, _, k in srv.admission_log]
    assert kinds.count("admit") == 5 and "wait" in kinds


def test_request_that_can_never_fit_is_refused():
    small = _req(0, 20, 0.0)
    big = _req(1, 400, 0.0)
    dev = FakeDevice(total=2 * serve.estimate_bytes(small))
    srv = _server(dev, slots=2)
    rep = srv.run([small, big])
    assert rep["failed"] == 1
    assert big.error and big.error.startswith("refused")
    assert small.error is None and small.steps == len(small.step_ms)


def test_late_arrivals_join_while_others_run():
    dev = FakeDevice(total=1 << 40)
    early = [_req(k, 20, 0.0, steps=40) for k in range(2)]
    late = _req(2, 20, 0.02, steps=5)
    rep = _server(dev, slots=4).run(early + [late])
    assert rep["failed"] == 0
    # the late one was admitted before the early ones finished
    assert late.admitted < min(r.finished for r in early)
    assert late.admitted >= 0.02


class FakeBatch:
    """Records the members of every tick; fail_at: fails the ticks with
    that many members."""

    def __init__(self, fail_at=None, adapt_fails=()):
        self.ticks = []
        self.adapts = []
        self.fail_at = fail_at
        self.adapt_fails = set(adapt_fails)

    def set_graphs(self, enable):
        self.graphs = enable

    def adapt(self, sims, errors="raise"):
        self.adapts.append([s.name for s in sims])
        out = []
        for s in sims:
            if s.name in self.adapt_fails:
                out.append((4, "split children exceed the capacity"))
            else:
                s.n += 1          # one more particle per adaptation
                out.append({"n_after": s.n})
        return out

    def step(self, sims, want_time=False):
        self.ticks.append([s.name for s in sims])
        time.sleep(0.001)
        if self.fail_at is not None and len(sims) == self.fail_at:
            raise RuntimeError("device error")

    def close(self):
        self.closed = True


class FakeSim:
    def __init__(self, name, n):
        self.name, self.n = name, n

    def info(self):
        return {"n": self.n}


def test_batch_stepper_members_join_and_leave():
    fb = FakeBatch()
    st = serve.BatchStepper(4, 0, batch=fb)
    reqs = [serve.Request(k, None, steps, adapt_every=0)
            for k, steps in enumerate((6, 3, 9))]
    sims = [FakeSim("s%d" % k, 100 * (k + 1)) for k in range(3)]

    def run(k, delay):
        time.sleep(delay)
        st.advance(sims[k], reqs[k])

    th = [threading.Thread(target=run, args=(k, 0.004 * k)) for k in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    st.close()
    assert fb.closed and fb.graphs is False
    for k, r in enumerate(reqs):
        # one latency per step, every step in a tick of its own
        assert len(r.step_ms) == r.steps
        assert r.particle_steps == r.steps * sims[k].n
        mine = [i for i, t in enumerate(fb.ticks) if sims[k].name in t]
        assert len(mine) == r.steps
        assert mine == list(range(mine[0], mine[0] + r.steps))   # consecutive
    assert max(len(t) for t in fb.ticks) <= 3
    assert sum(len(t) for t in fb.ticks) == 18


def test_batch_stepper_failure_reaches_every_member():
    fb = FakeBatch(fail_at=2)
    st = serve.BatchStepper(4, 0, batch=fb)
    # long enough that the second member joins while the first runs
    reqs = [serve.Request(k, None, 2000, adapt_every=0) for k in range(2)]
    sims = [FakeSim("a", 10), FakeSim("b", 20)]
    errs = []

    def run(k):
        try:
            st.advance(sims[k], reqs[k])
        except RuntimeError as e:
            errs.append(str(e))

    th = [threading.Thread(target=run, args=(k,)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    st.close()
    assert len(errs) == 2 and all("device error" in e for e in errs)
    assert all(r.error for r in reqs)


def test_batch_stepper_adapts_members_due_and_drops_failed_ones():
    """A member with adapt_every = k is adapted before its steps 0, k, 2k,
    ... (as run_alone does), in the tick's one adapt call; its particle
    count follows the adaptation.  A member whose adaptation fails leaves
    with its error; the others step on."""
    fb = FakeBatch(adapt_fails=("bad",))
    st = serve.BatchStepper(4, 0, batch=fb)
    reqs = [serve.Request(0, None, 6, adapt_every=2),
            serve.Request(1, None, 4, adapt_every=0),
            serve.Request(2, None, 5, adapt_every=1)]
    sims = [FakeSim("a", 100), FakeSim("b", 200), FakeSim("bad", 300)]
    errs = []

    def run(k):
        try:
            st.advance(sims[k], reqs[k])
        except RuntimeError as e:
            errs.append(str(e))

    th = [threading.Thread(target=run, args=(k,)) for k in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    st.close()
    assert len(errs) == 1 and "capacity" in errs[0]
    assert reqs[2].error and not reqs[0].error and not reqs[1].error
    a_adapts = [i for i, t in enumerate(fb.adapts) if "a" in t]
    assert len(a_adapts) == 3                      # before steps 0, 2, 4
    assert all("b" not in t for t in fb.adapts)
    assert all("bad" not in t for t in fb.ticks)   # never stepped
    assert len(reqs[0].step_ms) == 6 and len(reqs[1].step_ms) == 4
    # particle counts after each adaptation: 101, 101, 102, 102, 103, 103
    assert reqs[0].particle_steps == 2 * (101 + 102 + 103)
    assert reqs[1].particle_steps == 4 * 200


def test_batched_server_routes_adaptive_and_plain_requests_apart():
    """With batch=True the requests with adaptation go through one stepper
    and those without through the other, each request once."""
    made = []

    def make_stepper(k, stream):
        st = serve.BatchStepper(k, stream, batch=FakeBatch())
        made.append(st)
        return st

    def runner(req, stream, stepper):
        stepper.advance(FakeSim("r%d" % req.rid, 50), req)

    dev = FakeDevice(1 << 40)
    srv = serve.Server(slots=4, reserve=0, mem_info=dev.mem_info,
                       make_stream=lambda: (None, 0), batch=True,
                       make_stepper=make_stepper, batch_runner=runner)
    reqs = [serve.Request(k, wl.taylor_green(nx=8), 3 + k, adapt_every=k % 2,
                          arrival=0.001 * k) for k in range(6)]
    rep = srv.run(reqs)
    assert rep["failed"] == 0 and len(made) == 2
    plain, adaptive = made        # created for flags False, True
    seen_plain = {n for t in plain.batch.ticks for n in t}
    seen_adapt = {n for t in adaptive.batch.ticks for n in t}
    assert seen_plain == {"r0", "r2", "r4"} and seen_adapt == {"r1", "r3", "r5"}
    assert not plain.batch.adapts
    assert {n for t in adaptive.batch.adapts for n in t} == seen_adapt
    assert all(len(r.step_ms) == r.steps for r in reqs)
