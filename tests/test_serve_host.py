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
