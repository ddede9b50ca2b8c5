"""The force on the solid (sph_forces; section "Force computation", Eq.
force-sph) against the oracle on identical inputs: each wall particle's
pressure and viscous force and the totals, on a closed body in a jittered
lattice with random pressure and velocity fields; and the drag and lift
coefficients of the bench's cylinder set-up stay finite."""
import math

import numpy as np
import pytest

import oracle
from paper_2107_01276_gb300 import sph
from paper_2107_01276_gb300 import workloads as wl
from tests.helpers import cuda_ok, stream_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not cuda_ok():
        pytest.skip("no CUDA device")


def _case(seed):
    d = wl.ring_in_lattice(ds=0.05, jitter=0.2, seed=seed)
    fl = d["particles"]
    rng = np.random.default_rng(seed + 100)
    n = fl["x"].size
    fl["u"][:] = 1.0 + rng.normal(0, 0.1, n)
    fl["v"][:] = rng.normal(0, 0.1, n)
    fl["p"][:] = 2.0 + rng.normal(0, 0.5, n)
    return d


@pytest.mark.parametrize("precision,tol", [(sph.SPH_FP64, 1e-10),
                                           (sph.SPH_MIXED, 2e-5)])
def test_forces_parity(precision, tol):
    d = _case(7)
    fl, walls = d["particles"], d["walls"]
    nw = walls["x"].size
    P = sph.make_params(d["params"], precision=precision,
                        capacity=fl["x"].size)
    sim = sph.Simulation(P, stream_handle())
    sim.load(fl)
    sim.load(walls, kind=sph.SPH_WALL)
    got = sim.forces(per_wall=True)
    again = sim.forces()                 # no state change between calls
    sim.close()
    OP = oracle.params(**d["params"])
    oracle.set_walls(walls)
    try:
        ref = oracle.forces(OP, oracle.make_state(fl), nw)
    finally:
        oracle.set_walls(None)
    pw, rw = got["per_wall"], ref["per_wall"]
    for c in range(4):
        scale = np.abs(rw[:, c]).max()
        assert np.abs(pw[:, c] - rw[:, c]).max() <= tol * scale, c
    for k, c0 in (("fp", 0), ("fv", 2)):
        scale = np.abs(rw[:, c0:c0 + 2]).sum()
        assert np.abs(got[k] - ref[k]).max() <= tol * scale, k
        assert np.array_equal(got[k], again[k]), k


def test_forces_without_walls_are_zero():
    d = wl.taylor_green(nx=20)
    P = sph.make_params(d["params"], capacity=400)
    sim = sph.Simulation(P, stream_handle())
    sim.load(d["particles"])
    f = sim.forces()
    sim.close()
    assert np.all(f["fp"] == 0) and np.all(f["fv"] == 0)


def test_cylinder_coefficients_finite():
    """The bench's set-up (D/50 to D/2, background built, 12 adaptations):
    after a few steps from the impulsive start the coefficients are finite
    and the skin friction drags the body downstream."""
    d = wl.cylinder(Re=40.0)
    pr = d["params"]
    P = sph.make_params(pr, precision=sph.SPH_MIXED, capacity=400000)
    sim = sph.Simulation(P, stream_handle())
    sim.load(d["particles"])
    sim.load(d["walls"], kind=sph.SPH_WALL)
    sim.load(d["background"], kind=sph.SPH_BACKGROUND)
    sim.background()
    for _ in range(12):
        sim.adapt()
    for _ in range(5):
        sim.adapt()
        sim.step(1)
    f = sim.forces()
    c = sim.coefficients(1.0, d["D"])
    sim.close()
    assert all(math.isfinite(v) for v in c.values())
    assert c["cd_sf"] > 0
    # Eq. cdcl on the same state: the forces over rho0 U^2 D / 2
    q = 0.5 * pr["rho0"] * d["D"]
    assert c["cd_p"] == pytest.approx(f["fp"][0] / q, rel=1e-13)
    assert c["cd_sf"] == pytest.approx(f["fv"][0] / q, rel=1e-13)
    assert c["cl"] == pytest.approx(f["fp"][1] / q, rel=1e-13)
