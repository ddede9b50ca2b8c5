"""Parity of the background construction (sph_background, section 3.3)
and of the fluid vorticity (SPH_F_OMEGA) with the CPU oracle.

Inputs for every comparison come from the seeded generators or from the
oracle's own construction: the oracle runs the construction k iterations
from the initial lattice, and both sides then run one more iteration from
that state.  Decisions (marking, the Cr^3 test, the split threshold) are
FP64 with explicit rounding on both sides, so counts, ids and masses agree
exactly; sizes, h and positions agree to sum-order rounding."""
import math

import numpy as np
import pytest

import oracle
from paper_2107_01276_gb300 import sph
from tests.helpers import cuda_ok, stream_handle

pytestmark = pytest.mark.gpu

DS_MIN, DS_MAX, CR, HDX, LB, RAD = 0.1, 0.8, 1.2, 1.2, 16.0, 1.0
BG_FIELDS = ("x", "y", "h", "m", "ds")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not cuda_ok():
        pytest.skip("no CUDA device")


def _params():
    return dict(lo=(0.0, 0.0), hi=(LB, LB), periodic=(1, 1), rho0=1.0,
                cs=10.0, nu=0.01, hdx=HDX, Cr=CR, ds_min=DS_MIN, ds_max=DS_MAX)


def _solid():
    """Three rings of wall particles at ds_min inside a disk of radius 1."""
    xs, ys = [], []
    for k in range(3):
        r = RAD - (k + 0.5) * DS_MIN
        m = int(round(2 * np.pi * r / DS_MIN))
        a = 2 * np.pi * (np.arange(m) + 0.5 * (k % 2)) / m
        xs.append(LB / 2 + r * np.cos(a))
        ys.append(LB / 2 + r * np.sin(a))
    x, y = np.concatenate(xs), np.concatenate(ys)
    n = len(x)
    return {"x": x, "y": y, "h": np.full(n, HDX * DS_MIN),
            "m": np.full(n, DS_MIN * DS_MIN)}


def _lattice_bg():
    nx = int(round(LB / DS_MAX))
    g = (np.arange(nx) + 0.5) * LB / nx
    X, Y = np.meshgrid(g, g)
    n = X.size
    return {"x": X.ravel(), "y": Y.ravel(), "h": np.full(n, HDX * DS_MAX),
            "m": np.full(n, DS_MAX * DS_MAX), "ds": np.full(n, DS_MAX),
            "id": np.arange(n)}


def _fluid(nx=160, seed=3):
    """Fluid lattice over the box with a Taylor-Green velocity field."""
    rng = np.random.default_rng(seed)
    dx = LB / nx
    g = (np.arange(nx) + 0.5) * dx
    X, Y = np.meshgrid(g, g)
    x = (X.ravel() + rng.uniform(-0.05, 0.05, X.size) * dx) % LB
    y = (Y.ravel() + rng.uniform(-0.05, 0.05, X.size) * dx) % LB
    n = x.size
    k = 2 * np.pi / LB * 2
    return {"x": x, "y": y, "u": -np.cos(k * x) * np.sin(k * y),
            "v": np.sin(k * x) * np.cos(k * y), "p": np.zeros(n),
            "rho": 1.0 + 0.01 * rng.uniform(-1, 1, n),
            "m": np.full(n, dx * dx), "h": np.full(n, HDX * dx)}


@pytest.fixture(scope="module")
def oracle_stages():
    """Oracle background states after 0, 2 and 30 iterations."""
    P = oracle.params(**_params())
    B = oracle.bg_params(DS_MIN, DS_MAX, CR)
    b = oracle.make_bgset(_lattice_bg(), cap=100000)
    stages = {}
    nid = b["n"]
    for it in range(31):
        if it in (0, 2, 30):
            n = b["n"]
            stages[it] = {k: b[k][:n].copy() for k in BG_FIELDS + ("id",)}
        r, _, nid = oracle.bg_iteration(P, B, b, nid, _solid())
        assert r == 0
    return stages


def _one_iteration_both(state, fluid=None, vort_k=0.0, precision=sph.SPH_FP64):
    pr = _params()
    P = sph.make_params(pr, precision=precision, capacity=200000,
                        vort_k=vort_k, bg_capacity=200000)
    sim = sph.Simulation(P, stream_handle())
    if fluid is not None:
        sim.load(fluid)
    sim.load(_solid(), kind=sph.SPH_WALL)
    sim.load(state, kind=sph.SPH_BACKGROUND)
    g = sim.background(1)
    got = sim.read_background()
    order = np.argsort(got["id"], kind="stable")
    got = {k: v[order] for k, v in got.items()}
    OP = oracle.params(**pr)
    B = oracle.bg_params(DS_MIN, DS_MAX, CR, vort_k=vort_k)
    b = oracle.make_bgset(state, cap=200000)
    nid = int(state["id"].max()) + 1
    fl = None
    if fluid is not None:
        st = oracle.make_state(fluid)
        fl = dict(fluid, phi=np.abs(oracle.vorticity(OP, st)))
    r, o, _ = oracle.bg_iteration(OP, B, b, nid, _solid(), fl)
    assert r == 0
    n = b["n"]
    order = np.argsort(b["id"][:n], kind="stable")
    ref = {k: b[k][:n][order] for k in BG_FIELDS + ("id",)}
    sim.close()
    return g, o, got, ref


@pytest.mark.parametrize("stage", [0, 2, 30])
def test_one_iteration_parity(oracle_stages, stage):
    g, o, got, ref = _one_iteration_both(oracle_stages[stage])
    for k in ("n_before", "n_marked", "n_vort", "n_split", "n_after"):
        assert g[k] == o[k], (k, g, o)
    assert np.array_equal(got["id"], ref["id"])
    assert np.array_equal(got["m"], ref["m"])
    assert np.abs(got["ds"] / ref["ds"] - 1).max() < 1e-12
    assert np.abs(got["h"] / ref["h"] - 1).max() < 1e-12
    for k in ("x", "y"):
        d = got[k] - ref[k]
        d -= LB * np.round(d / LB)
        assert np.abs(d).max() < 1e-12 * LB, k


def test_vorticity_parity():
    fl = _fluid()
    P = sph.make_params(_params(), precision=sph.SPH_FP64, capacity=len(fl["x"]))
    sim = sph.Simulation(P, stream_handle())
    sim.load(fl)
    w = sim.read("omega")
    ids = sim.read("id")
    got = np.empty_like(w)
    got[ids] = w
    ref = oracle.vorticity(oracle.params(**_params()), oracle.make_state(fl))
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    sim.close()


def test_vorticity_marking_parity(oracle_stages):
    g, o, got, ref = _one_iteration_both(oracle_stages[30], fluid=_fluid(),
                                         vort_k=0.5)
    assert o["n_vort"] > 0
    for k in ("n_marked", "n_vort", "n_split", "n_after"):
        assert g[k] == o[k], (k, g, o)
    assert np.array_equal(got["id"], ref["id"])
    assert np.abs(got["ds"] / ref["ds"] - 1).max() < 1e-12


@pytest.mark.parametrize("stage", [0, 2, 30])
def test_one_iteration_parity_mixed(oracle_stages, stage):
    """A mixed context's construction sums the shifting step's pairs in
    FP32 (state in FP64); marking, sizes, splits and the h-smoothing stay
    FP64.  One iteration from the oracle's states: counts, ids, masses and
    sizes as in FP64 (they are decided before the first shift); h and
    positions within the FP32 pair sums' rounding."""
    g, o, got, ref = _one_iteration_both(oracle_stages[stage],
                                         precision=sph.SPH_MIXED)
    for k in ("n_before", "n_marked", "n_vort", "n_split", "n_after"):
        assert g[k] == o[k], (k, g, o)
    assert np.array_equal(got["id"], ref["id"])
    assert np.array_equal(got["m"], ref["m"])
    assert np.abs(got["ds"] / ref["ds"] - 1).max() < 1e-12
    assert np.abs(got["h"] / ref["h"] - 1).max() < 1e-5
    for k in ("x", "y"):
        d = got[k] - ref[k]
        d -= LB * np.round(d / LB)
        assert np.abs(d).max() < 2e-5 * HDX * DS_MAX, k


@pytest.mark.parametrize("precision", [sph.SPH_FP64, sph.SPH_MIXED])
def test_full_construction_invariants(precision):
    """The whole construction (3 ceil(log 8 / log 1.2) = 36 iterations) on
    the GPU: sizes in [ds_min, ds_max], ds_min next to the solid, sizes of
    neighbours within Cr^3, about N_r neighbours, mass conserved, size
    growing outward; and the same particle count and per-ring sizes as the
    oracle's construction, for both precisions."""
    P = sph.make_params(_params(), precision=precision, capacity=1000,
                        bg_capacity=200000)
    sim = sph.Simulation(P, stream_handle())
    sim.load(_solid(), kind=sph.SPH_WALL)
    bg0 = _lattice_bg()
    sim.load(bg0, kind=sph.SPH_BACKGROUND)
    g = sim.background()
    assert g["iterations"] == 36
    b = sim.read_background()
    sim.close()
    n = len(b["x"])
    assert abs(math.fsum(b["m"]) - math.fsum(bg0["m"])) <= 1e-13 * LB * LB
    assert b["ds"].min() >= DS_MIN and b["ds"].max() <= DS_MAX
    # neighbour sets of the result, r < 3 max(h_i, h_j), by a k-d tree
    from scipy.spatial import cKDTree
    pts = np.stack([b["x"], b["y"]], axis=1) % LB
    tree = cKDTree(pts, boxsize=LB)
    own = tree.query_ball_point(pts, r=3.0 * b["h"])
    sets = [set(o) for o in own]
    for i, o in enumerate(own):
        for j in o:
            sets[j].add(i)
    N = np.array([len(t) for t in sets])
    assert 44 <= np.median(N) <= 52
    ratio = np.array([b["ds"][list(t)].max() / b["ds"][list(t)].min() for t in sets])
    assert ratio.max() <= CR ** 3 * (1 + 1e-12)
    r = np.hypot(b["x"] - LB / 2, b["y"] - LB / 2)
    edges = [1.0, 1.3, 1.6, 2.0, 2.5, 3.0, 4.0, 5.0, 7.0]
    med = [np.median(b["ds"][(r >= a) & (r < c)]) for a, c in zip(edges, edges[1:])]
    assert all(y >= x for x, y in zip(med, med[1:]))
    assert med[0] == DS_MIN and med[-1] == DS_MAX
    # oracle's own construction from the same lattice
    OP = oracle.params(**_params())
    ob = oracle.make_bgset(bg0, cap=200000)
    r0, _, _ = oracle.bg_build(OP, oracle.bg_params(DS_MIN, DS_MAX, CR), ob, _solid())
    assert r0 == 0
    assert abs(n - ob["n"]) <= 0.01 * ob["n"]
    ro = np.hypot(ob["x"][:ob["n"]] - LB / 2, ob["y"][:ob["n"]] - LB / 2)
    med_o = [np.median(ob["ds"][:ob["n"]][(ro >= a) & (ro < c)])
             for a, c in zip(edges, edges[1:])]
    assert np.allclose(med, med_o, rtol=0.15)


def test_background_every_n_bg_adapt_calls(oracle_stages):
    """n_bg = 2: the second sph_adapt call runs one background iteration
    first; the background then equals one explicit sph_background(1)."""
    fl = _fluid(nx=80)
    state = oracle_stages[2]
    outs = []
    for mode in ("hook", "explicit"):
        P = sph.make_params(_params(), precision=sph.SPH_FP64, capacity=200000,
                            bg_capacity=200000, n_bg=2 if mode == "hook" else 0)
        sim = sph.Simulation(P, stream_handle())
        sim.load(fl)
        sim.load(_solid(), kind=sph.SPH_WALL)
        sim.load(state, kind=sph.SPH_BACKGROUND)
        if mode == "hook":
            sim.adapt()
            assert sim.info()["n_bg"] == len(state["x"])
            sim.adapt()
        else:
            sim.background(1)
        b = sim.read_background()
        order = np.argsort(b["id"])
        outs.append({k: v[order] for k, v in b.items()})
        sim.close()
    for k in ("id", "m", "ds", "h", "x", "y"):
        assert np.array_equal(outs[0][k], outs[1][k]), k


def test_background_errors():
    P = sph.make_params(_params(), precision=sph.SPH_FP64, capacity=100,
                        bg_capacity=500)
    sim = sph.Simulation(P, stream_handle())
    with pytest.raises(sph.SphError) as e:
        sim.background(1)
    assert e.value.status == sph.SPH_ESTATE
    sim.load(_solid(), kind=sph.SPH_WALL)
    sim.load(_lattice_bg(), kind=sph.SPH_BACKGROUND)
    with pytest.raises(sph.SphError) as e:
        sim.background(5)                      # splits exceed 500
    assert e.value.status == sph.SPH_ECAPACITY
    # the context stays usable and holds the completed iterations
    b = sim.read_background()
    assert 400 <= len(b["x"]) <= 500
    sim.close()
    P = sph.make_params(_params(), precision=sph.SPH_FP64, capacity=100, Cr=1.0)
    sim = sph.Simulation(P, stream_handle())
    sim.load(_lattice_bg(), kind=sph.SPH_BACKGROUND)
    with pytest.raises(sph.SphError) as e:
        sim.background(1)
    assert e.value.status == sph.SPH_EINVAL
    sim.close()


def test_moving_body_update_parity(oracle_stages):
    """A moving body (section 3.3: the background is updated by single
    iterations as the solid moves): the context first holds the walls at
    their old position, they are reloaded 0.5 further along x, and one
    iteration from the oracle's state runs against the moved walls.  Both
    sides take the same decisions: counts, ids and masses exact."""
    pr = _params()
    OP = oracle.params(**pr)
    B = oracle.bg_params(DS_MIN, DS_MAX, CR)
    b = oracle.make_bgset(oracle_stages[30], cap=200000)
    nid = int(oracle_stages[30]["id"].max()) + 1
    r, _, nid = oracle.bg_iteration(OP, B, b, nid, _solid())
    assert r == 0
    n = b["n"]
    s1 = {k: b[k][:n].copy() for k in BG_FIELDS + ("id",)}
    moved = _solid()
    moved["x"] = moved["x"] + 0.5
    r, o, _ = oracle.bg_iteration(OP, B, b, nid, moved)
    assert r == 0 and o["n_marked"] > 0
    n = b["n"]
    order = np.argsort(b["id"][:n], kind="stable")
    ref = {k: b[k][:n][order] for k in BG_FIELDS + ("id",)}

    P = sph.make_params(pr, precision=sph.SPH_FP64, capacity=1000,
                        bg_capacity=200000)
    sim = sph.Simulation(P, stream_handle())
    sim.load(_solid(), kind=sph.SPH_WALL)
    sim.load(s1, kind=sph.SPH_BACKGROUND)
    sim.load(moved, kind=sph.SPH_WALL)          # the body moved
    g = sim.background(1)
    got = sim.read_background()
    sim.close()
    order = np.argsort(got["id"], kind="stable")
    got = {k: v[order] for k, v in got.items()}
    for k in ("n_marked", "n_split", "n_after"):
        assert g[k] == o[k], (k, g, o)
    assert np.array_equal(got["id"], ref["id"])
    assert np.array_equal(got["m"], ref["m"])
    assert np.abs(got["ds"] / ref["ds"] - 1).max() < 1e-12


def test_background_follows_a_moving_body():
    """The paper's moving-solid experiment in small: after the full
    construction the body moves 0.05 per step for 20 steps with one
    background iteration per step; ds_min then sits at the body's new
    surface and the old position has coarsened."""
    P = sph.make_params(_params(), precision=sph.SPH_FP64, capacity=1000,
                        bg_capacity=400000)
    sim = sph.Simulation(P, stream_handle())
    sim.load(_solid(), kind=sph.SPH_WALL)
    sim.load(_lattice_bg(), kind=sph.SPH_BACKGROUND)
    sim.background()
    body = _solid()
    for _ in range(20):
        body["x"] = body["x"] + 0.05
        sim.load(body, kind=sph.SPH_WALL)
        sim.background(1)
    b = sim.read_background()
    sim.close()
    c_new = (LB / 2 + 1.0, LB / 2)
    r_new = np.hypot(b["x"] - c_new[0], b["y"] - c_new[1])
    near = (r_new > RAD) & (r_new < RAD + 0.3)
    assert near.sum() > 0 and np.median(b["ds"][near]) == DS_MIN
    # behind the body, where its surface was, sizes have grown
    r_old = np.hypot(b["x"] - (LB / 2 - 1.0), b["y"] - LB / 2)
    behind = (r_old < 0.3)
    assert behind.sum() > 0 and np.median(b["ds"][behind]) > DS_MIN
