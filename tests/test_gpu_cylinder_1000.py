"""Parity at the shape of the solution-adaptive cylinder run (Re 1000,
spacing D/1000 at the wall to D/4, 1:250, vorticity adaptivity): the
fluid initialised from the graded ring background (~52k particles, 12.5k
wall particles), cell keys of every particle, and for a random sample the
neighbour sets and the right-hand side with the walls, evaluated one by
one by the oracle.  Then the run itself: adaptation and PEC steps with a
vorticity-driven background iteration keep mass and stay finite."""
import math

import numpy as np
import pytest

import oracle
from paper_2107_01276_gb300 import sph
from paper_2107_01276_gb300 import workloads as wl
from tests.helpers import FP64_TOL, MIXED_TOL, cuda_ok, norm, stream_handle
from tests.test_gpu_fullsize import RHS_FIELDS, _sparse_csr

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def c1000():
    if not cuda_ok():
        pytest.skip("no CUDA device")
    d = wl.cylinder(Re=1000.0, ds_min_over_D=1 / 1000, ds_max_over_D=1 / 4,
                    background="rings", fluid="rings")
    d["params"] = dict(d["params"], vort_k=0.05, n_bg=4)
    return d


def _oracle_sampled(d, sample, dt):
    pt, walls = d["particles"], d["walls"]
    P = oracle.params(**d["params"])
    n = len(pt["x"])
    xs = lambda idx: (pt["x"][idx], pt["y"][idx], pt["h"][idx])
    o1, n1 = oracle.neighbors_cross(P, *xs(sample), pt["x"], pt["y"], pt["h"])
    U = np.unique(np.concatenate([sample, n1]))
    oU, nU = oracle.neighbors_cross(P, *xs(U), pt["x"], pt["y"], pt["h"])
    off, nbr = _sparse_csr(n, U, oU, nU)
    oracle.set_walls(walls)
    try:
        oracle.wall_bc_store(P, oracle.make_state(pt))
        with np.errstate(all="ignore"):
            a = oracle.pass_a(P, pt["x"], pt["y"], pt["h"], pt["m"], pt["p"],
                              off, nbr)
            offs, nbrs = _sparse_csr(n, sample, o1, n1)
            b = oracle.pass_b(P, dt, pt["x"], pt["y"], pt["h"], pt["m"],
                              pt["p"], pt["u"], pt["v"], offs, nbrs, a)
    finally:
        oracle.set_walls(None)
    out = {k: v[sample] for k, v in b.items()}
    for k in ("rho", "beta", "pavg", "drx", "dry", "nnb", "s_rho", "s_beta",
              "s_pavg", "s_drx", "s_dry"):
        out[k] = a[k][sample]
    return (o1, n1), out


@pytest.mark.parametrize("precision,tol", [(sph.SPH_MIXED, MIXED_TOL),
                                           (sph.SPH_FP64, FP64_TOL)])
def test_sampled_parity_with_walls(c1000, precision, tol):
    d = c1000
    pt = d["particles"]
    n = len(pt["x"])
    P = sph.make_params(d["params"], precision=precision, capacity=n)
    sim = sph.Simulation(P, stream_handle())
    sim.load(pt)
    sim.load(d["walls"], kind=sph.SPH_WALL)
    sim.rhs()
    ids = sim.read("id")
    pos = np.empty(n, np.int64)
    pos[ids] = np.arange(n)
    key = sim.read("cellkey")
    okey, _ = oracle.cell_keys(oracle.params(**d["params"]),
                               sim.info()["c0"], pt["x"], pt["y"], pt["h"])
    assert np.array_equal(key[pos], okey)
    rng = np.random.default_rng(23)
    sample = np.sort(rng.choice(n, 200, replace=False))
    dt = oracle.dt(oracle.params(**d["params"]), pt["h"])
    (o1, n1), ref = _oracle_sampled(d, sample, dt)
    off = sim.read("neigh_off")
    nid = sim.read("neigh_id")
    for k, i in enumerate(sample):
        p = pos[i]
        assert np.array_equal(np.sort(nid[off[p]:off[p + 1]]),
                              n1[o1[k]:o1[k + 1]]), i
    got = {f: sim.read(f)[pos[sample]] for f in RHS_FIELDS}
    assert np.array_equal(sim.read("nnb")[pos[sample]], ref["nnb"])
    for f in RHS_FIELDS:
        e = norm(got[f], ref[f], ref["s_" + f])
        assert e <= tol, (f, e)
    sim.close()


def test_solution_adaptive_run(c1000):
    """Adaptation + PEC steps with a background iteration every 4th call
    (vorticity marking on): mass conserved to rounding through splits and
    merges, the finest fluid mass at the wall stays near rho0 ds_min^2, all
    fields finite."""
    d = c1000
    pt = d["particles"]
    P = sph.make_params(d["params"], precision=sph.SPH_MIXED,
                        capacity=2_000_000, bg_capacity=2_000_000)
    sim = sph.Simulation(P, stream_handle())
    sim.load(pt)
    sim.load(d["walls"], kind=sph.SPH_WALL)
    sim.load(d["background"], kind=sph.SPH_BACKGROUND)
    m0 = math.fsum(pt["m"])
    for _ in range(12):
        g = sim.adapt()
        assert abs(g["mass_after"] - g["mass_before"]) <= 1e-12 * m0
        sim.step(1)
    m = sim.read("m")
    assert abs(math.fsum(m) - m0) <= 1e-11 * m0
    for f in ("x", "y", "u", "v", "p", "h"):
        assert np.all(np.isfinite(sim.read(f))), f
    x, y = sim.read("x"), sim.read("y")
    cx, cy = 7.5 * d["D"], 7.5 * d["D"]
    near = np.hypot(x - cx, y - cy) < 0.5 * d["D"] + 0.01
    ds_min = d["params"]["ds_min"]
    assert near.sum() > 1000
    assert np.median(m[near]) <= 1.05 * 1000.0 * ds_min ** 2
    sim.close()
