"""Parity of the dummy-wall boundary (section 2.2) on the GPU with the
oracle: right-hand sides and PEC steps next to a wall, and the cylinder
workload (walls, background, adaptation) at the size of configs[1]."""
import math

import numpy as np
import pytest

import oracle
from paper_2107_01276_gb300 import sph
from paper_2107_01276_gb300 import workloads as wl
from tests.helpers import FP64_TOL, MIXED_TOL, by_id, cuda_ok, norm, \
    stream_handle

pytestmark = pytest.mark.gpu
RHS_FIELDS = ("rho", "beta", "pavg", "drx", "dry", "dpdt", "dudt", "dvdt")
STATE = ("x", "y", "u", "v", "p", "rho", "m", "h", "mmin", "mmax")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not cuda_ok():
        pytest.skip("no CUDA device")


def _sim(d, precision, cap=None, walls=True, bg=False):
    n = len(d["particles"]["x"])
    P = sph.make_params(d["params"], precision=precision,
                        capacity=cap or max(n, 1))
    sim = sph.Simulation(P, stream_handle())
    sim.load(d["particles"])
    if walls:
        sim.load(d["walls"], kind=sph.SPH_WALL)
    if bg:
        sim.load(d["background"], kind=sph.SPH_BACKGROUND)
    return sim


def _oracle_rhs(d, particles=None):
    P = oracle.params(**d["params"])
    pt = particles if particles is not None else d["particles"]
    st = oracle.make_state(pt)
    dt = oracle.dt(P, pt["h"][:len(pt["x"])])
    oracle.set_walls(d["walls"])
    try:
        return oracle.rhs(P, dt, st)
    finally:
        oracle.set_walls(None)


@pytest.mark.parametrize("precision,tol", [(sph.SPH_FP64, FP64_TOL),
                                           (sph.SPH_MIXED, MIXED_TOL)])
def test_rhs_parity_next_to_a_wall(precision, tol):
    d = wl.half_plane_walls()
    sim = _sim(d, precision)
    sim.rhs()
    got = by_id(sim, list(RHS_FIELDS) + ["nnb"])
    ref = _oracle_rhs(d)
    assert np.array_equal(got["nnb"], ref["nnb"])
    for f in RHS_FIELDS:
        assert norm(got[f], ref[f], ref["s_" + f]) <= tol, f
    sim.close()


def test_pec_steps_next_to_a_wall():
    d = wl.half_plane_walls(seed=3)
    sim = _sim(d, sph.SPH_FP64)
    t = sim.step(5)
    got = by_id(sim, ["x", "y", "u", "v", "p"])
    P = oracle.params(**d["params"])
    st = oracle.make_state(d["particles"])
    oracle.set_walls(d["walls"])
    try:
        tr = oracle.step(P, st, 5)
    finally:
        oracle.set_walls(None)
    assert abs(t - tr) <= 1e-15 * tr
    n = st["n"]
    for f in ("u", "v", "p"):
        sc = np.abs(st[f][:n]).max()
        assert np.abs(got[f] - st[f][:n]).max() <= 1e-10 * sc, f
    Lx = d["params"]["hi"][0]
    dxs = got["x"] - st["x"][:n]
    dxs -= Lx * np.round(dxs / Lx)
    assert np.abs(dxs).max() <= 1e-10 * d["dx"]
    sim.close()


@pytest.fixture(scope="module")
def cyl_refined():
    """configs[1]-shaped cylinder: coarse fluid refined by repeated
    sph_adapt against the graded background, with the oracle checking one
    adaptation call on identical inputs."""
    if not cuda_ok():
        pytest.skip("no CUDA device")
    d = wl.cylinder()
    sim = _sim(d, sph.SPH_FP64, cap=200000, bg=True)
    P = oracle.params(**d["params"])
    stats = []
    for call in range(12):
        before = by_id(sim, list(STATE))
        nid = sim.info()["next_id"]
        g = sim.adapt()
        stats.append(g)
        if call in (0, 6):
            st = oracle.make_state(before, cap=200000)
            oracle.set_walls(d["walls"])
            try:
                r, o, _ = oracle.adapt(P, st, bg=d["background"],
                                       next_id=nid)
            finally:
                oracle.set_walls(None)
            assert r == 0
            assert (g["n_split"], g["n_merged"], g["n_after"]) == \
                (o["n_split"], o["n_merged"], o["n_after"]), call
    return d, sim, stats


def test_cylinder_refines_and_conserves_mass(cyl_refined):
    d, sim, stats = cyl_refined
    n = sim.info()["n"]
    assert 5000 < n < 40000
    m0 = math.fsum(d["particles"]["m"])
    assert abs(math.fsum(sim.read("m")) - m0) <= 1e-12 * m0
    # the last calls split little: the refinement has settled
    assert stats[-1]["n_split"] < 0.05 * n
    # finest particles sit next to the cylinder
    x, y, m = sim.read("x"), sim.read("y"), sim.read("m")
    r = np.hypot(x - 15.0, y - 15.0)
    near, far = r < 1.3, r > 8.0
    assert np.median(m[near]) < 0.02 * np.median(m[far])


@pytest.mark.parametrize("precision,tol", [(sph.SPH_FP64, FP64_TOL),
                                           (sph.SPH_MIXED, MIXED_TOL)])
def test_cylinder_rhs_parity(cyl_refined, precision, tol):
    d, sim, _ = cyl_refined
    state = by_id(sim, list(STATE))
    P = sph.make_params(d["params"], precision=precision, capacity=200000)
    s2 = sph.Simulation(P, stream_handle())
    s2.load(state)
    s2.load(d["walls"], kind=sph.SPH_WALL)
    s2.rhs()
    got = by_id(s2, list(RHS_FIELDS) + ["nnb"])
    ref = _oracle_rhs(d, particles=state)
    assert np.array_equal(got["nnb"], ref["nnb"])
    for f in RHS_FIELDS:
        assert norm(got[f], ref[f], ref["s_" + f]) <= tol, f
    s2.close()
