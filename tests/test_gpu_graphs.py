"""sph_step replayed as captured CUDA graphs: on a stream of its own the
library captures a step once per buffer assignment and replays it; the
states it reaches equal those of the launch-by-launch step bit for bit,
for both precisions, with walls, and across a change of the particle set
(a new capture)."""
import gc

import numpy as np
import pytest
import torch

from paper_2107_01276_gb300 import sph
from paper_2107_01276_gb300 import workloads as wl
from tests.helpers import by_id, cuda_ok

pytestmark = pytest.mark.gpu
FIELDS = ["x", "y", "u", "v", "p", "rho", "h", "m"]


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not cuda_ok():
        pytest.skip("no CUDA device")


@pytest.fixture(autouse=True)
def _no_other_contexts():
    # graphs are used only while a context is the only live one
    gc.collect()


def _run(d, precision, graphs, steps, stream, cap=None):
    n = len(d["particles"]["x"])
    P = sph.make_params(d["params"], precision=precision, capacity=cap or n)
    s = sph.Simulation(P, stream.cuda_stream)
    s.set_tuning(graphs=graphs)
    s.load(d["particles"])
    if "walls" in d:
        s.load(d["walls"], kind=sph.SPH_WALL)
    t = None
    for _ in range(steps):
        t = s.step(1, want_time=False)
    t = s.step(1)
    out = by_id(s, FIELDS)
    gs = s.info()["graph_steps"]
    s.close()
    return t, out, gs


@pytest.mark.parametrize("precision", [sph.SPH_FP64, sph.SPH_MIXED])
def test_graph_steps_equal_launch_by_launch(precision):
    d = wl.perturbed(nx=120, ny=100, h_ratio=3.0, seed=41)
    st = torch.cuda.Stream()
    t0, a, g0 = _run(d, precision, False, 12, st)
    t1, b, g1 = _run(d, precision, True, 12, st)
    assert g0 == 0 and g1 >= 8          # replayed after the first steps
    assert t0 == t1
    for f in FIELDS:
        assert np.array_equal(a[f], b[f]), f


def test_graph_steps_with_walls_and_reload():
    d = wl.ring_in_lattice(ds=0.05, jitter=0.1, seed=9)
    fl = d["particles"]
    rng = np.random.default_rng(10)
    fl["u"][:] = 0.5 + rng.normal(0, 0.05, fl["x"].size)
    st = torch.cuda.Stream()
    res = []
    for graphs in (False, True):
        n = fl["x"].size
        P = sph.make_params(d["params"], precision=sph.SPH_MIXED, capacity=n)
        s = sph.Simulation(P, st.cuda_stream)
        s.set_tuning(graphs=graphs)
        s.load(fl)
        s.load(d["walls"], kind=sph.SPH_WALL)
        for _ in range(6):
            s.step(1, want_time=False)
        # a new particle set mid-run: the captured graphs no longer apply
        state = by_id(s, FIELDS + ["id"])
        s.load({k: state[k] for k in FIELDS})
        for _ in range(6):
            s.step(1, want_time=False)
        res.append((by_id(s, FIELDS), s.info()["graph_steps"]))
        s.close()
    (a, g0), (b, g1) = res
    assert g0 == 0 and g1 >= 6
    for f in FIELDS:
        assert np.array_equal(a[f], b[f]), f
