"""Pins of the oracle's adaptive refinement (section 3): split geometry and
bookkeeping, merge rules and the merged smoothing length in closed form,
mass / momentum / centroid conservation, the shift and Taylor correction on
fields with known gradients, the h update, and the background resolution
against an independent k-d tree search."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2107_01276_gb300 import workloads as wl

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "paper_constants.json")))
ALPHA = GOLD["split_alpha"]["value"]
EPS = GOLD["split_eps"]["value"]


def _state(parts, cap=None):
    return oracle.make_state(parts, cap=cap)


def _one(x=0.5, y=0.5, m=1.0, h=0.1, mmax=0.5, pid=0, **kw):
    d = dict(x=[x], y=[y], u=[kw.get("u", 0.3)], v=[kw.get("v", -0.2)],
             p=[kw.get("p", 7.0)], rho=[kw.get("rho", 1.01)], m=[m], h=[h],
             mmin=[0.1], mmax=[mmax], id=[pid])
    return {k: np.asarray(v, dtype=np.int64 if k == "id" else float)
            for k, v in d.items()}


def _P(**kw):
    return oracle.params(**dict(dict(lo=(0, 0), hi=(1, 1), periodic=(0, 0)),
                                **kw))


# ------------------------------------------------------------------ split --
def test_split_geometry_and_bookkeeping():
    st = _state(_one(), cap=16)
    cnt, nid = oracle.split(_P(), st, next_id=100)
    assert cnt == 1 and nid == 106 and st["n"] == 7
    n = 7
    x, y = st["x"][:n], st["y"][:n]
    ids = st["id"][:n]
    assert ids[0] == 0 and list(ids[1:]) == list(range(100, 106))
    # centre child keeps the parent's place
    assert x[0] == 0.5 and y[0] == 0.5
    # six children on the circle of radius eps h at angles k pi / 3
    r = np.hypot(x[1:] - 0.5, y[1:] - 0.5)
    assert np.allclose(r, EPS * 0.1, rtol=1e-14, atol=0)
    ang = np.arctan2(y[1:] - 0.5, x[1:] - 0.5)
    exp = np.array([k * math.pi / 3 for k in range(6)])
    dang = (ang - exp + math.pi) % (2 * math.pi) - math.pi
    assert np.abs(dang).max() < 1e-13
    assert np.allclose(st["h"][:n], ALPHA * 0.1, rtol=1e-15, atol=0)
    m = st["m"][:n]
    assert np.allclose(m[1:], 1.0 / 7.0, rtol=1e-15, atol=0)
    assert abs(math.fsum(m) - 1.0) <= 1e-16
    # centre of mass stays at the parent (hexagon symmetry)
    assert abs(math.fsum(m * x) - 0.5) < 1e-15
    assert abs(math.fsum(m * y) - 0.5) < 1e-15
    for k, v in (("u", 0.3), ("v", -0.2), ("p", 7.0), ("rho", 1.01),
                 ("mmin", 0.1), ("mmax", 0.5)):
        assert np.all(st[k][:n] == v)


def test_split_child_ids_follow_parent_id_order():
    a, b, c = _one(x=0.2, pid=10), _one(x=0.5, pid=3, mmax=2.0), \
        _one(x=0.8, pid=5)
    parts = {k: np.concatenate([a[k], b[k], c[k]]) for k in a}
    st = _state(parts, cap=32)
    cnt, nid = oracle.split(_P(), st, next_id=50)
    assert cnt == 2 and nid == 62 and st["n"] == 15
    ids = st["id"][:15]
    # id 5 (rank 0) gets 50..55, id 10 (rank 1) gets 56..61
    x = st["x"][:15]
    near = lambda x0: set(ids[np.abs(x - x0) < 0.1]) - {10, 5, 3}
    assert near(0.8) == set(range(50, 56))
    assert near(0.2) == set(range(56, 62))


def test_split_refuses_over_capacity_and_respects_no_limit():
    st = _state(_one(), cap=6)
    cnt, nid = oracle.split(_P(), st, next_id=1)
    assert cnt == -1 and st["n"] == 1 and nid == 1
    st = _state(_one(mmax=0.0), cap=16)       # m_max <= 0: no limit
    cnt, _ = oracle.split(_P(), st, next_id=1)
    assert cnt == 0 and st["n"] == 1


# ------------------------------------------------------------------ merge --
def _pair(xa, xb, ha=0.1, hb=0.1, ma=1.0, mb=1.0, mmax=5.0, ids=(0, 1),
          ya=0.5, yb=0.5):
    return {"x": np.array([xa, xb]), "y": np.array([ya, yb]),
            "u": np.array([1.0, -2.0]), "v": np.array([0.5, 0.25]),
            "p": np.array([3.0, 7.0]), "rho": np.array([1.0, 1.2]),
            "m": np.array([ma, mb]), "h": np.array([ha, hb]),
            "mmin": np.array([0.0, 0.0]), "mmax": np.array([mmax, mmax]),
            "id": np.array(ids, dtype=np.int64)}


def test_merged_h_closed_forms():
    """Eq. merged-h with coincident particles: W(0, h) = W(0, 1)/h^2 in 2-D,
    so equal h gives h back, and unequal h gives sqrt(2 ha^2 hb^2 /
    (ha^2 + hb^2))."""
    st = _state(_pair(0.5, 0.5, ha=0.1, hb=0.1))
    assert oracle.merge_round(_P(), st) == 1
    assert st["n"] == 1 and abs(st["h"][0] - 0.1) < 1e-16
    ha, hb = 0.1, 0.13
    st = _state(_pair(0.5, 0.5, ha=ha, hb=hb))
    assert oracle.merge_round(_P(), st) == 1
    exp = math.sqrt(2 * ha * ha * hb * hb / (ha * ha + hb * hb))
    assert abs(st["h"][0] - exp) < 1e-15


def test_merge_conserves_mass_momentum_and_centroid():
    st = _state(_pair(0.50, 0.53, ma=1.0, mb=3.0, ids=(7, 4)))
    assert oracle.merge_round(_P(), st) == 1
    assert st["n"] == 1 and st["id"][0] == 4          # smaller id kept
    assert st["m"][0] == 4.0
    assert abs(st["x"][0] - (0.50 * 1 + 0.53 * 3) / 4) < 1e-15
    assert abs(st["u"][0] - (1.0 * 1 - 2.0 * 3) / 4) < 1e-15
    assert abs(st["p"][0] - (3.0 * 1 + 7.0 * 3) / 4) < 1e-15
    assert abs(st["rho"][0] - (1.0 * 1 + 1.2 * 3) / 4) < 1e-15


def test_merge_across_periodic_boundary_uses_nearest_image():
    P = _P(periodic=(1, 1))
    st = _state(_pair(0.99, 0.01, ma=1.0, mb=1.0))
    assert oracle.merge_round(P, st) == 1
    assert abs(st["x"][0] - 0.0) < 1e-15 or abs(st["x"][0] - 1.0) < 1e-15


def test_merge_rules():
    # too far: r >= (h_a + h_b)/2
    st = _state(_pair(0.5, 0.61))
    assert oracle.merge_round(_P(), st) == 0 and st["n"] == 2
    # too heavy: m_a + m_b >= max(m_max)
    st = _state(_pair(0.5, 0.52, ma=2.5, mb=2.5, mmax=5.0))
    assert oracle.merge_round(_P(), st) == 0
    # one of them is to be split (m > m_max)
    pr = _pair(0.5, 0.52, ma=1.0, mb=1.0, mmax=5.0)
    pr["mmax"][1] = 0.9
    assert oracle.merge_round(_P(), _state(pr)) == 0
    # no limit (m_max <= 0) never merges
    assert oracle.merge_round(_P(), _state(_pair(0.5, 0.52, mmax=0.0))) == 0


def test_merge_only_mutually_closest_pairs():
    """A at 0, B at 0.02, C at 0.06: A and B are each other's closest and
    merge; C's closest is B, whose closest is A, so C stays."""
    parts = {"x": np.array([0.5, 0.52, 0.56]), "y": np.full(3, 0.5),
             "u": np.zeros(3), "v": np.zeros(3), "p": np.zeros(3),
             "rho": np.ones(3), "m": np.ones(3), "h": np.full(3, 0.1),
             "mmin": np.zeros(3), "mmax": np.full(3, 5.0),
             "id": np.arange(3, dtype=np.int64)}
    st = _state(parts)
    assert oracle.merge_round(_P(), st) == 1
    assert st["n"] == 2 and sorted(st["id"][:2]) == [0, 2]


def test_merge_tie_breaks_on_smaller_id():
    """B equidistant from A and C: B's closest is the one with the smaller
    id."""
    parts = {"x": np.array([0.48, 0.50, 0.52]), "y": np.full(3, 0.5),
             "u": np.zeros(3), "v": np.zeros(3), "p": np.zeros(3),
             "rho": np.ones(3), "m": np.ones(3), "h": np.full(3, 0.1),
             "mmin": np.zeros(3), "mmax": np.full(3, 5.0),
             "id": np.array([9, 1, 4], dtype=np.int64)}
    st = _state(parts)
    assert oracle.merge_round(_P(), st) == 1
    assert sorted(st["id"][:2]) == [1, 9]          # B(1) merged with C(4)


# ------------------------------------------------------- shift and Taylor --
def test_shift_is_a_no_op_on_a_periodic_lattice():
    tg = wl.taylor_green(nx=24, hdx=1.2)
    P = oracle.params(**tg["params"])
    st = _state(tg["particles"])
    n = st["n"]
    x0, u0 = st["x"][:n].copy(), st["u"][:n].copy()
    sc = oracle.shift_compute(P, st)
    assert np.abs(sc["drx"]).max() < 1e-15 * tg["dx"]
    oracle.shift_round(P, st)
    assert np.abs(st["x"][:n] - x0).max() < 1e-15
    assert np.abs(st["u"][:n] - u0).max() < 1e-12


def test_taylor_gradient_of_linear_field():
    """grad phi = sum V_j (phi_j - phi_i) grad W on a lattice recovers the
    gradient of a linear field in the interior (full support of i and of
    every j)."""
    tg = wl.taylor_green(nx=40, hdx=1.2)
    pr = dict(tg["params"], periodic=(0, 0))
    P = oracle.params(**pr)
    pt = dict(tg["particles"])
    pt["u"] = 2.0 * pt["x"] - 3.0 * pt["y"]
    pt["v"] = 0.5 * pt["y"]
    pt["p"] = -pt["x"]
    st = _state(pt)
    sc = oracle.shift_compute(P, st)
    dx = tg["dx"]
    inner = ((pt["x"] > 8 * dx) & (pt["x"] < 1 - 8 * dx) &
             (pt["y"] > 8 * dx) & (pt["y"] < 1 - 8 * dx))
    for k, v in (("gux", 2.0), ("guy", -3.0), ("gvx", 0.0), ("gvy", 0.5),
                 ("gpx", -1.0), ("gpy", 0.0)):
        assert np.abs(sc[k][inner] - v).max() < 3e-3 * 3.0, k


def test_taylor_correction_follows_the_shift():
    """Jittered lattice, linear u: after a shift round u' stays close to the
    field at the new positions, much closer than the uncorrected u."""
    tg = wl.taylor_green(nx=40, hdx=1.2, jitter=0.25, seed=4)
    pr = dict(tg["params"], periodic=(0, 0))
    P = oracle.params(**pr)
    pt = dict(tg["particles"])
    pt["u"] = 2.0 * pt["x"] + 1.0 * pt["y"]
    st = _state(pt)
    n = st["n"]
    u_old = st["u"][:n].copy()
    oracle.shift_round(P, st)
    dx = tg["dx"]
    x, y = st["x"][:n], st["y"][:n]
    inner = (x > 8 * dx) & (x < 1 - 8 * dx) & (y > 8 * dx) & (y < 1 - 8 * dx)
    exact = 2.0 * x + y
    err_c = np.abs(st["u"][:n] - exact)[inner].max()
    err_0 = np.abs(u_old - exact)[inner].max()
    assert err_0 > 1e-3 * dx
    assert err_c < 0.2 * err_0          # the uncorrected operator is ~10 % off on a jittered set


# --------------------------------------------------------------- h update --
@pytest.mark.parametrize("hdx", [1.0, 1.2])
def test_h_update_on_uniform_lattice(hdx):
    """Equal masses m = rho0 dx^2 and rho ~ rho0 give h = hdx dx."""
    tg = wl.taylor_green(nx=30, hdx=hdx)
    P = oracle.params(**tg["params"])
    st = _state(tg["particles"])
    n = st["n"]
    st["h"][:n] *= 1.1                     # start away from the optimum
    oracle.h_update(P, st)
    assert np.allclose(st["h"][:n], hdx * tg["dx"], rtol=2e-3, atol=0)


# ------------------------------------------------- background resolution --
def test_background_resolution_against_kdtree():
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(9)
    nb, nf = 300, 500
    bg = {"x": rng.uniform(0, 1, nb), "y": rng.uniform(0, 1, nb),
          "h": rng.uniform(0.03, 0.08, nb), "ds": rng.uniform(0.01, 0.05, nb)}
    fl = {"x": rng.uniform(0, 1, nf), "y": rng.uniform(0, 1, nf),
          "u": np.zeros(nf), "v": np.zeros(nf), "p": np.zeros(nf),
          "rho": np.ones(nf), "m": np.full(nf, 1e-3),
          "h": rng.uniform(0.005, 0.05, nf)}
    P = _P(rho0=1000.0)
    st = _state(fl)
    oracle.bg_resolution(P, st, bg)
    tb = cKDTree(np.stack([bg["x"], bg["y"]], 1))
    for i in range(nf):
        q = (fl["x"][i], fl["y"][i])
        cand = tb.query_ball_point(q, 3 * max(fl["h"][i], bg["h"].max()))
        ok = [b for b in cand if math.dist(q, (bg["x"][b], bg["y"][b])) <
              3 * max(fl["h"][i], bg["h"][b])]
        if ok:
            mref = 1000.0 * min(bg["ds"][b] ** 2 for b in ok)
        else:
            mref = 1000.0 * bg["ds"][tb.query(q)[1]] ** 2
        assert abs(st["mmax"][i] - 1.05 * mref) <= 1e-15 * mref
        assert abs(st["mmin"][i] - 0.5 * mref) <= 1e-15 * mref


# ------------------------------------------------------- whole adaptation --
def _refine_case():
    """Coarse perturbed lattice; the background asks for half the spacing
    in the left half of the box."""
    d = wl.perturbed(nx=30, ny=30, h_ratio=1.0, jitter=0.1, hdx=1.2,
                     periodic=(1, 1), seed=12)
    dx = d["dx"]
    g = (np.arange(60) + 0.5) / 60
    X, Y = np.meshgrid(g, g, indexing="xy")
    bg = {"x": X.ravel(), "y": Y.ravel(), "h": np.full(X.size, 1.2 / 60)}
    bg["ds"] = np.where(bg["x"] < 0.5, 0.5 * dx, dx)
    return d, bg


def test_adapt_conserves_mass_and_refines():
    d, bg = _refine_case()
    P = oracle.params(**d["params"])
    st = _state(d["particles"], cap=20000)
    m0 = math.fsum(st["m"][:st["n"]])
    r, stats, nid = oracle.adapt(P, st, bg=bg)
    n = st["n"]
    assert r == 0 and stats["n_split"] > 0 and n > stats["n_before"]
    assert abs(math.fsum(st["m"][:n]) - m0) <= 1e-14 * m0
    assert len(set(st["id"][:n])) == n                 # ids stay unique
    # repeated adaptation settles: the last call splits (almost) nothing
    for _ in range(4):
        r, stats, nid = oracle.adapt(P, st, bg=bg, next_id=nid)
    n = st["n"]
    assert abs(math.fsum(st["m"][:n]) - m0) <= 1e-14 * m0
    assert stats["n_split"] <= 0.02 * n
    # the background reaches 3 h_b = 0.06 beyond the left half (and
    # across the periodic wrap)
    left = (st["x"][:n] > 0.1) & (st["x"][:n] < 0.4)
    right = (st["x"][:n] > 0.65) & (st["x"][:n] < 0.85)
    assert np.median(st["m"][:n][left]) < 0.6 * np.median(st["m"][:n][right])
