"""Pins of the oracle's background construction (section 3.3) and of the
vorticity it uses for solution adaptivity: hand-worked size-rule cases,
brute-force marking, the fixed point of Eq. h-smoothing on a lattice, zero
shift on a uniform lattice, the iteration count, vorticity of closed-form
flows, and the invariants a finished construction must satisfy (sizes in
[ds_min, ds_max], ds_min next to the solid, neighbouring sizes within a
factor Cr^3, mass conserved, about N_r neighbours)."""
import math

import numpy as np
import pytest

import oracle


def _P(L=10.0, periodic=(1, 1), **kw):
    return oracle.params(lo=(0.0, 0.0), hi=(L, L), periodic=periodic, **kw)


def _set(x, y, h, ds, m=None):
    n = len(x)
    return oracle.make_bgset({"x": np.asarray(x, float), "y": np.asarray(y, float),
                              "h": np.broadcast_to(np.asarray(h, float), (n,)).copy(),
                              "ds": np.asarray(ds, float),
                              "m": np.ones(n) if m is None else np.asarray(m, float)},
                             cap=8 * n + 8)


def _lattice(nx, L, h, periodic=True):
    g = (np.arange(nx) + 0.5) * L / nx
    X, Y = np.meshgrid(g, g)
    return X.ravel(), Y.ravel()


def test_iteration_count():
    # 3 ceil(log(25) / log(1.08)) = 3 * 42; 3 ceil(log 4 / log 1.2) = 3 * 8
    assert oracle.bg_iterations(oracle.bg_params(0.04, 1.0, 1.08)) == 126
    assert oracle.bg_iterations(oracle.bg_params(0.1, 0.4, 1.2)) == 24


def test_class_search_equals_brute_force():
    rng = np.random.default_rng(5)
    for periodic in ((1, 1), (0, 1), (0, 0)):
        P = _P(L=4.0, periodic=periodic)
        n = 700
        x, y = rng.uniform(0, 4.0, n), rng.uniform(0, 4.0, n)
        h = 0.01 * np.exp(rng.uniform(0, math.log(30.0), n))
        a = oracle.neighbors(P, x, y, h, method="brute")
        b = oracle.neighbors_classes(P, x, y, h)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_size_rule_hand_cases():
    P = _P()
    B = oracle.bg_params(0.01, 10.0, 1.1)
    # three mutual neighbours
    x, y = [1.0, 1.5, 2.0], [1.0, 1.0, 1.0]
    b = _set(x, y, 1.0, [1.0, 1.0, 1.0])
    oracle.bg_size(P, B, b, np.zeros(3, np.uint8))
    assert np.all(b["ds"][:3] == 1.1)                 # ratio 1 < Cr^3: Cr lo
    # particle 0 sees {1, 1} -> 1.1; the others see {0.04, 1}: ratio 25 >=
    # Cr^3 -> geometric mean 0.2.  Jacobi: 0 reads the old sizes.
    b = _set(x, y, 1.0, [0.04, 1.0, 1.0])
    oracle.bg_size(P, B, b, np.zeros(3, np.uint8))
    assert b["ds"][0] == pytest.approx(1.1, rel=1e-15)
    assert b["ds"][1:3] == pytest.approx([0.2, 0.2], rel=1e-14)
    # {1.0, 1.2}: ratio 1.2 < 1.331 -> 1.1 x 1.0
    b = _set(x, y, 1.0, [5.0, 1.0, 1.2])
    oracle.bg_size(P, B, b, np.zeros(3, np.uint8))
    assert b["ds"][0] == pytest.approx(1.1, rel=1e-15)
    # a marked particle keeps its size and still counts as a neighbour
    b = _set(x, y, 1.0, [0.01, 1.0, 1.0])
    oracle.bg_size(P, B, b, np.array([1, 0, 0], np.uint8))
    assert b["ds"][0] == 0.01
    assert b["ds"][1] == pytest.approx(math.sqrt(0.01), rel=1e-14)
    # clamped to ds_max; an isolated particle keeps its size
    B2 = oracle.bg_params(0.01, 1.0, 1.1)
    b = _set([1.0, 1.5, 8.0], [1.0, 1.0, 8.0], 0.3, [1.0, 1.0, 0.5])
    oracle.bg_size(P, B2, b, np.zeros(3, np.uint8))
    assert list(b["ds"][:3]) == [1.0, 1.0, 0.5]


def test_marking_is_brute_force_range_test():
    rng = np.random.default_rng(2)
    P = _P(L=6.0)
    n, ns = 400, 60
    x, y = rng.uniform(0, 6, n), rng.uniform(0, 6, n)
    h = rng.uniform(0.05, 0.4, n)
    sx, sy = rng.uniform(2, 4, ns), rng.uniform(2, 4, ns)
    sh = np.full(ns, 0.05)
    b = _set(x, y, h, np.full(n, 0.8))
    B = oracle.bg_params(0.05, 0.8, 1.1)
    mark = oracle.bg_mark(P, B, b, {"x": sx, "y": sy, "h": sh})

    def within(ax, ay, ah, bx_, by_, bh_):
        dx = ax[:, None] - bx_[None, :]
        dy = ay[:, None] - by_[None, :]
        dx -= 6.0 * np.round(dx / 6.0)
        dy -= 6.0 * np.round(dy / 6.0)
        R = 3.0 * np.maximum(ah[:, None], bh_[None, :])
        return dx * dx + dy * dy < R * R

    near = within(x, y, h, sx, sy, sh).any(axis=1)
    assert 0 < near.sum() < n
    assert np.array_equal(mark == 1, near)
    assert np.all(b["ds"][:n][near] == 0.05) and np.all(b["ds"][:n][~near] == 0.8)
    # vorticity marking: fluid particles with phi; threshold k max phi
    nf = 300
    fx, fy = rng.uniform(0, 6, nf), rng.uniform(0, 6, nf)
    fh = np.full(nf, 0.1)
    phi = rng.uniform(0, 1, nf) ** 4
    B = oracle.bg_params(0.05, 0.8, 1.1, vort_k=0.3)
    b = _set(x, y, h, np.full(n, 0.8))
    mark = oracle.bg_mark(P, B, b, {"x": sx, "y": sy, "h": sh},
                          {"x": fx, "y": fy, "h": fh, "phi": phi})
    inr = within(x, y, h, fx, fy, fh)
    pb = np.where(inr, phi[None, :], 0.0).max(axis=1)
    hot = (pb > 0.3 * phi.max()) & ~near
    assert hot.sum() > 0
    assert np.array_equal(mark == 2, hot)
    assert np.array_equal(mark == 1, near)


def test_split_conserves_mass_and_copies_size():
    P = _P(split_alpha=0.9, split_eps=0.4)
    b = _set([2.0, 5.0, 7.0], [2.0, 5.0, 7.0], 0.6, [0.1, 1.0, 0.5],
             m=[1.0, 1.0, 0.2])
    # m > 1.05 rho0 ds^2: particle 0 (1 > 0.0105) only
    r, nid = oracle.bg_split(P, b, 3)
    assert r == 1 and b["n"] == 9 and nid == 9
    assert math.fsum(b["m"][:9]) == pytest.approx(2.2, rel=1e-15)
    assert np.all(b["ds"][3:9] == 0.1)
    assert list(b["id"][3:9]) == [3, 4, 5, 6, 7, 8]
    assert b["h"][0] == pytest.approx(0.54) and np.all(b["h"][3:9] == b["h"][0])
    d = np.hypot(b["x"][3:9] - 2.0, b["y"][3:9] - 2.0)
    assert np.allclose(d, 0.4 * 0.6, rtol=1e-14)


def test_h_smoothing_fixed_point_on_a_lattice():
    # square lattice, spacing 1: 45 points lie within r < 3 h for 9 h^2 in
    # (13, 16]; with N_r = 45 the lattice h is a fixed point
    L = 20.0
    x, y = _lattice(20, L, 1.3)
    n = len(x)
    P = _P(L=L)
    b = _set(x, y, 1.3, np.ones(n))
    oracle.bg_hsmooth(P, oracle.bg_params(0.1, 1.0, 1.1, Nr=45.0), b)
    assert np.allclose(b["h"][:n], 1.3, rtol=1e-14, atol=0)
    # fewer neighbours than N_r: h grows; more: h shrinks
    b = _set(x, y, 1.3, np.ones(n))
    oracle.bg_hsmooth(P, oracle.bg_params(0.1, 1.0, 1.1, Nr=48.0), b)
    assert np.all(b["h"][:n] > 1.3)
    b = _set(x, y, 1.3, np.ones(n))
    oracle.bg_hsmooth(P, oracle.bg_params(0.1, 1.0, 1.1, Nr=30.0), b)
    assert np.all(b["h"][:n] < 1.3)


def test_h_smoothing_converges_to_about_Nr_neighbours():
    L = 20.0
    x, y = _lattice(20, L, 1.0)
    n = len(x)
    P = _P(L=L)
    b = _set(x, y, 0.9, np.ones(n))
    B = oracle.bg_params(0.1, 1.0, 1.1)
    for _ in range(30):
        oracle.bg_hsmooth(P, B, b)
    off, _ = oracle.neighbors(P, b["x"][:n], b["y"][:n], b["h"][:n])
    N = np.diff(off)
    assert 45 <= N.min() and N.max() <= 57


def test_shift_leaves_a_uniform_lattice_in_place():
    L = 12.0
    x, y = _lattice(24, L, 0.6)
    n = len(x)
    P = _P(L=L)
    b = _set(x, y, 0.6, np.full(n, 0.5), m=np.full(n, 0.25))
    oracle.bg_shift(P, b)
    assert np.abs(b["x"][:n] - x).max() < 1e-13
    assert np.abs(b["y"][:n] - y).max() < 1e-13


def test_shift_separates_a_close_pair():
    L = 12.0
    x, y = _lattice(24, L, 0.6)
    x = np.append(x, x[300] + 0.05)
    y = np.append(y, y[300])
    n = len(x)
    P = _P(L=L)
    b = _set(x, y, 0.6, np.full(n, 0.5), m=np.full(n, 0.25))
    oracle.bg_shift(P, b)
    assert b["x"][300] < x[300] and b["x"][n - 1] > x[n - 1]


def _fluid_lattice(nx, L, hdx, u, v):
    dx = L / nx
    g = (np.arange(nx) + 0.5) * dx
    X, Y = np.meshgrid(g, g)
    x, y = X.ravel(), Y.ravel()
    n = len(x)
    f = {"x": x, "y": y, "u": u(x, y), "v": v(x, y), "m": np.full(n, dx * dx),
         "h": np.full(n, hdx * dx), "rho": np.ones(n)}
    return f, dx


def test_vorticity_of_rigid_rotation_and_taylor_green():
    # rigid rotation about the box centre: omega = 2 Omega in the interior
    L, Om = 1.0, 0.7
    f, dx = _fluid_lattice(40, L, 1.2, lambda x, y: -Om * (y - 0.5),
                           lambda x, y: Om * (x - 0.5))
    P = oracle.params(lo=(0, 0), hi=(L, L), periodic=(0, 0), hdx=1.2)
    st = oracle.make_state(f)
    w = oracle.vorticity(P, st)
    inner = (np.abs(f["x"] - 0.5) < 0.3) & (np.abs(f["y"] - 0.5) < 0.3)
    assert np.abs(w[inner] / (2 * Om) - 1).max() < 2e-3
    # the same operator as the Taylor-correction gradients (which use the
    # summation density for V_j): omega = dv/dx - du/dy
    g = oracle.shift_compute(P, st)
    st["rho"][:len(f["x"])] = g["rho"]
    w2 = oracle.vorticity(P, st)
    assert np.abs(w2 - (g["gvx"] - g["guy"])).max() < 1e-12 * np.abs(w2).max()
    # Taylor-Green: omega = 4 pi U cos(2 pi x) cos(2 pi y), periodic box
    U = 1.0
    k = 2 * np.pi
    f, dx = _fluid_lattice(50, 1.0, 1.2,
                           lambda x, y: -U * np.cos(k * x) * np.sin(k * y),
                           lambda x, y: U * np.sin(k * x) * np.cos(k * y))
    P = oracle.params(lo=(0, 0), hi=(1, 1), periodic=(1, 1), hdx=1.2)
    w = oracle.vorticity(P, oracle.make_state(f))
    ex = 2 * k * U * np.cos(k * f["x"]) * np.cos(k * f["y"])
    assert np.abs(w - ex).max() < 2e-2 * np.abs(ex).max()


@pytest.fixture(scope="module")
def small_build():
    """A disk of solid particles (3 rings at ds_min) in a periodic box; the
    background starts as a ds_max lattice over the whole box."""
    ds_min, ds_max, Cr, hdx, Lb, R = 0.1, 0.8, 1.2, 1.2, 16.0, 1.0
    P = oracle.params(lo=(0, 0), hi=(Lb, Lb), periodic=(1, 1), rho0=1.0,
                      hdx=hdx)
    xs, ys = [], []
    for k in range(3):
        r = R - (k + 0.5) * ds_min
        m = int(round(2 * np.pi * r / ds_min))
        a = 2 * np.pi * (np.arange(m) + 0.5 * (k % 2)) / m
        xs.append(Lb / 2 + r * np.cos(a))
        ys.append(Lb / 2 + r * np.sin(a))
    solid = {"x": np.concatenate(xs), "y": np.concatenate(ys)}
    solid["h"] = np.full(len(solid["x"]), hdx * ds_min)
    x, y = _lattice(20, Lb, hdx * ds_max)
    n = len(x)
    b = oracle.make_bgset({"x": x, "y": y, "h": np.full(n, hdx * ds_max),
                           "m": np.full(n, ds_max * ds_max),
                           "ds": np.full(n, ds_max)}, cap=100000)
    B = oracle.bg_params(ds_min, ds_max, Cr)
    r, stats, _ = oracle.bg_build(P, B, b, solid)
    assert r == 0 and len(stats) == 36
    return P, B, solid, b, n * ds_max * ds_max


def test_finished_background_invariants(small_build):
    P, B, solid, b, mass0 = small_build
    n = b["n"]
    x, y, h, ds, m = (b[k][:n] for k in ("x", "y", "h", "ds", "m"))
    assert abs(math.fsum(m) - mass0) <= 1e-13 * mass0
    assert ds.min() >= B.ds_min and ds.max() <= B.ds_max
    off, nbr = oracle.neighbors(P, x, y, h)
    N = np.diff(off)
    assert 44 <= np.median(N) <= 52
    ratio = np.array([ds[nbr[off[i]:off[i + 1]]].max() /
                      ds[nbr[off[i]:off[i + 1]]].min() for i in range(n)])
    assert ratio.max() <= B.Cr ** 3 * (1 + 1e-12)
    # next to the solid: the finest size; far away: the coarsest
    mark = oracle.bg_mark(P, B, oracle.make_bgset(
        {k: b[k][:n] for k in oracle.BG_FIELDS}), solid)
    assert np.all(ds[mark == 1] == B.ds_min)
    r = np.hypot(x - 8.0, y - 8.0)
    assert np.all(ds[r > 7.0] == B.ds_max)
    # size grows outward: medians over rings are non-decreasing
    edges = [1.0, 1.3, 1.6, 2.0, 2.5, 3.0, 4.0, 5.0, 7.0]
    med = [np.median(ds[(r >= a) & (r < c)]) for a, c in zip(edges, edges[1:])]
    assert all(b2 >= a2 for a2, b2 in zip(med, med[1:]))
    assert med[0] == B.ds_min and med[-1] == B.ds_max
