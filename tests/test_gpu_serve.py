"""The serving loop on the GPU: simulations of different kinds and sizes
admitted together, overlapping on the device on their own streams, each
ending in exactly the state it reaches alone (every context is independent
and its kernels are deterministic), and a latency report."""
import numpy as np
import pytest

from paper_2107_01276_gb300 import serve
from paper_2107_01276_gb300 import workloads as wl
from tests.helpers import cuda_ok, stream_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not cuda_ok():
        pytest.skip("no CUDA device")


def _requests():
    return [
        serve.Request(0, wl.taylor_green(nx=40, Re=100.0), 20, adapt_every=0),
        serve.Request(1, wl.gresho_chan(nx=40), 20, adapt_every=2, refine=2,
                      arrival=0.01),
        serve.Request(2, wl.taylor_green_adaptive(nx=40), 20, adapt_every=4,
                      refine=3, arrival=0.02),
        serve.Request(3, wl.cylinder(Re=200.0, ds_min_over_D=1 / 25.0), 10,
                      adapt_every=1, refine=6, arrival=0.0,
                      bg_capacity=200000),
        serve.Request(4, wl.taylor_green(nx=70, Re=400.0), 20, adapt_every=0,
                      arrival=0.03),
    ]


def test_each_result_is_the_same_alone_and_in_the_mix():
    alone = [serve.run_alone(r, stream_handle()) for r in _requests()]
    mix = _requests()
    srv = serve.Server(slots=4, keep_final=True)
    rep = srv.run(mix)
    assert rep["failed"] == 0, [r.error for r in mix]
    kinds = [k for _, _, k in srv.admission_log]
    assert kinds.count("admit") == len(mix)
    for a, b in zip(alone, mix):
        assert a.particle_steps == b.particle_steps
        for f, v in a.final.items():
            assert np.array_equal(v, b.final[f]), (a.rid, f)
    assert rep["steps"] == sum(r.steps for r in mix)
    assert 0 < rep["step_ms_p50"] <= rep["step_ms_p99"]
    assert rep["particle_steps_per_s"] > 0


def test_batched_steps_match_alone():
    """With batch=True the requests step together (sph_batch_step, joining
    and leaving as they are admitted and finish), the adaptive one through
    the adaptive requests' stepper (sph_batch_adapt, then sph_batch_step);
    with their team sizes set, each ends bit for bit where it ends alone."""
    def reqs():
        return [
            serve.Request(0, wl.taylor_green(nx=40, Re=100.0), 12, adapt_every=0, team=4),
            serve.Request(1, wl.taylor_green(nx=70, Re=400.0), 20, adapt_every=0,
                          arrival=0.02, team=4),
            serve.Request(2, wl.gresho_chan(nx=40), 10, adapt_every=2, refine=2,
                          arrival=0.01),
            serve.Request(3, wl.taylor_green(nx=55, Re=250.0), 16, adapt_every=0,
                          arrival=0.03, team=4),
        ]
    alone = [serve.run_alone(r, stream_handle()) for r in reqs()]
    mix = reqs()
    srv = serve.Server(slots=4, keep_final=True, batch=True)
    rep = srv.run(mix)
    assert rep["failed"] == 0, [r.error for r in mix]
    for a, b in zip(alone, mix):
        assert a.particle_steps == b.particle_steps
        assert len(b.step_ms) == b.steps
        for f, v in a.final.items():
            assert np.array_equal(v, b.final[f]), (a.rid, f)
