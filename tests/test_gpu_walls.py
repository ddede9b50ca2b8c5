"""Parity of the dummy-wall boundary (section 2.2) on the GPU with the
oracle: right-hand sides and PEC steps next to a wall, and the cylinder
workload (walls, background, adaptation) at the bench's size (D/50 to D/2).  Every
oracle input comes from the seeded generators or from the oracle itself."""
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


def _snapshot(st):
    n = st["n"]
    out = {k: st[k][:n].copy() for k in STATE}
    out["id"] = st["id"][:n].copy()
    return out


@pytest.fixture(scope="module")
def cyl_oracle():
    """The oracle's own refinement of the cylinder's coarse lattice against
    the C_r-graded ring background: its states before adaptation calls 0
    and 6 and after call 6."""
    d = wl.cylinder(background="rings")
    P = oracle.params(**d["params"])
    st = oracle.make_state(d["particles"], cap=200000)
    nid = st["n"]
    states = {}
    oracle.set_walls(d["walls"])
    try:
        for call in range(7):
            if call in (0, 6):
                states[call] = _snapshot(st)
            r, _, nid = oracle.adapt(P, st, bg=d["background"], next_id=nid)
            assert r == 0
    finally:
        oracle.set_walls(None)
    states["final"] = _snapshot(st)
    return d, states


@pytest.mark.parametrize("call", [0, 6])
def test_cylinder_adapt_parity(cyl_oracle, call):
    """One sph_adapt call from the oracle's state before call `call`:
    counts, ids and masses equal the oracle's (FP64 decisions)."""
    d, states = cyl_oracle
    state = states[call]
    sim = _sim(dict(d, particles=state), sph.SPH_FP64, cap=200000, bg=True)
    g = sim.adapt()
    got = by_id(sim, ["m", "mmax"])
    sim.close()
    P = oracle.params(**d["params"])
    st = oracle.make_state(state, cap=200000)
    oracle.set_walls(d["walls"])
    try:
        r, o, _ = oracle.adapt(P, st, bg=d["background"],
                               next_id=int(state["id"].max()) + 1)
    finally:
        oracle.set_walls(None)
    assert r == 0
    assert (g["n_split"], g["n_merged"], g["n_after"]) == \
        (o["n_split"], o["n_merged"], o["n_after"])
    n = st["n"]
    order = np.argsort(st["id"][:n])
    assert np.array_equal(got["id"], st["id"][:n][order])
    assert np.array_equal(got["m"], st["m"][:n][order])
    assert np.array_equal(got["mmax"], st["mmax"][:n][order])


@pytest.fixture(scope="module")
def cyl_refined():
    """The bench-sized cylinder (D/50 at the wall, D/2 far away) refined on the GPU alone: the coarse
    lattice through 12 sph_adapt calls against the ring background."""
    if not cuda_ok():
        pytest.skip("no CUDA device")
    d = wl.cylinder(background="rings")
    sim = _sim(d, sph.SPH_FP64, cap=200000, bg=True)
    stats = [sim.adapt() for _ in range(12)]
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
def test_cylinder_rhs_parity(cyl_oracle, precision, tol):
    """Right-hand side at the oracle's refined cylinder state."""
    d, states = cyl_oracle
    state = states["final"]
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


def test_cylinder_constructed_background():
    """The cylinder set-up as the bench runs it: the ds_max lattice refined by
    the full construction (3 ceil(log 25 / log 1.08) = 126 iterations) on
    the GPU: ds_min next to the cylinder, ds_max far away, sizes growing
    outward, mass of the background conserved."""
    d = wl.cylinder()
    assert d["construct_background"]
    sim = _sim(d, sph.SPH_MIXED, cap=200000, bg=True)
    g = sim.background()
    assert g["iterations"] == 126
    b = sim.read_background()
    sim.close()
    m0 = math.fsum(d["background"]["m"])
    assert abs(math.fsum(b["m"]) - m0) <= 1e-12 * m0
    pr = d["params"]
    assert b["ds"].min() >= pr["ds_min"] and b["ds"].max() <= pr["ds_max"]
    r = np.hypot(b["x"] - 15.0, b["y"] - 15.0)
    edges = [1.0, 1.2, 1.5, 2.0, 3.0, 5.0, 8.0, 12.0]
    med = [np.median(b["ds"][(r >= a) & (r < c)]) for a, c in zip(edges, edges[1:])]
    assert all(y >= x for x, y in zip(med, med[1:]))
    assert med[0] == pr["ds_min"] and med[-1] == pr["ds_max"]
