"""Failure paths, all triggered from the host with no GPU fault: a
non-finite pressure in a loaded state and a particle faster than the mixed
step's neighbour-list skin allows are reported as SPH_ENONFINITE, once,
and the context steps on normally after a clean state is loaded; a
checkpoint written with sph_read and loaded into a fresh context continues
the run bit for bit.

The non-finite case runs on the mixed path only: there a step builds its
lists once, from the loaded (finite) positions, and the non-finite rates
reach positions only after that build; the rebuild of the next call starts
from the clean state loaded in between."""
import numpy as np
import pytest

from paper_2107_01276_gb300 import sph
from paper_2107_01276_gb300 import workloads as wl
from tests.helpers import cuda_ok, stream_handle

pytestmark = pytest.mark.gpu

STATE = ("x", "y", "u", "v", "p", "rho", "m", "h", "mmin", "mmax")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not cuda_ok():
        pytest.skip("no CUDA device")


def _sim(d, precision, cap=None):
    n = len(d["particles"]["x"])
    P = sph.make_params(d["params"], precision=precision, capacity=cap or n)
    s = sph.Simulation(P, stream_handle())
    s.load(d["particles"])
    return s


def _state(sim):
    out = {k: sim.read(k) for k in STATE}
    out["id"] = sim.read("id")
    return out


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in STATE + ("id",))


def test_nonfinite_pressure_reported_once_then_usable():
    d = wl.taylor_green(nx=32, jitter=0.1, seed=4)
    bad = {k: v.copy() for k, v in d["particles"].items()}
    bad["p"][17] = np.nan
    sim = _sim(dict(d, particles=bad), sph.SPH_MIXED)
    with pytest.raises(sph.SphError) as e:
        sim.step(1)
    assert e.value.status == sph.SPH_ENONFINITE
    assert "non-finite" in str(e.value)
    # a clean state: steps as a fresh context does, no error carried over
    sim.load(d["particles"])
    sim.step(3)
    ref = _sim(d, sph.SPH_MIXED)
    ref.step(3)
    assert _same(_state(sim), _state(ref))
    sim.close()
    ref.close()


def test_skin_overrun_reported_then_usable():
    """One particle at 100 (U_ref + c_s = 11): the predictor moves it about
    a smoothing length, far beyond the 0.15 h the mixed step's list skin
    covers (and far inside the periodic box)."""
    d = wl.taylor_green(nx=32, jitter=0.1, seed=5)
    fast = {k: v.copy() for k, v in d["particles"].items()}
    fast["u"][40] = 100.0
    sim = _sim(dict(d, particles=fast), sph.SPH_MIXED)
    with pytest.raises(sph.SphError) as e:
        sim.step(1)
    assert e.value.status == sph.SPH_ENONFINITE
    assert "skin" in str(e.value)
    sim.load(d["particles"])
    sim.step(2)   # no error: the report was cleared with the new state
    ref = _sim(d, sph.SPH_MIXED)
    ref.step(2)
    assert _same(_state(sim), _state(ref))
    sim.close()
    ref.close()


@pytest.mark.parametrize("precision", [sph.SPH_FP64, sph.SPH_MIXED])
@pytest.mark.parametrize("case", ["tgv", "graded"])
def test_checkpoint_restore_bit_identical(case, precision):
    """k steps, every state field read (rows in the context's current
    order, ids included), loaded into a fresh context; k more steps on both
    give identical states and times."""
    d = (wl.taylor_green(nx=40, jitter=0.1, seed=6) if case == "tgv"
         else wl.graded_strip(n_target=20000, ratio=16.0))
    a = _sim(d, precision)
    t_a = a.step(4)
    ck = _state(a)
    b_d = dict(d, particles=ck)
    b = _sim(b_d, precision, cap=len(ck["x"]))
    ta2 = a.step(4)
    tb2 = b.step(4)
    assert ta2 - t_a == pytest.approx(tb2, rel=1e-14)
    assert _same(_state(a), _state(b))
    a.close()
    b.close()


def test_rejected_load_keeps_the_state():
    """A fluid set refused by the device-side checks (here one particle
    outside the box) leaves the context's state, ids and time untouched:
    the next steps are those of a context that never saw it."""
    d = wl.taylor_green(nx=32, jitter=0.1, seed=9)
    a = _sim(d, sph.SPH_MIXED)
    b = _sim(d, sph.SPH_MIXED)
    a.step(2)
    b.step(2)
    before = _state(a)
    bad = {k: v.copy() for k, v in d["particles"].items()}
    bad["x"][11] = 5.0
    with pytest.raises(sph.SphError) as e:
        a.load(bad)
    assert e.value.status == sph.SPH_EINVAL
    assert "outside the box" in str(e.value)
    assert _same(_state(a), before)
    ta, tb = a.step(3), b.step(3)
    assert ta == tb
    assert _same(_state(a), _state(b))
    a.close()
    b.close()
