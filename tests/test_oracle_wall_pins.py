"""Pins of the oracle's dummy-wall boundary (section 2.2): Shepard
extrapolation reproduces constants, walls restore the kernel support,
uniform states next to a wall stay force-free, a wall moving with the
stream adds nothing, and flow into a wall compresses."""
import numpy as np
import pytest

import oracle

DX = 0.02


def _half_plane(nx=30, ny=20, layers=4, hdx=1.2, rho0=1.0):
    """Fluid lattice y > 0 on an x-periodic strip; wall lattice of `layers`
    rows continuing it below y = 0."""
    gx = (np.arange(nx) + 0.5) * DX
    gy = (np.arange(ny) + 0.5) * DX
    X, Y = np.meshgrid(gx, gy, indexing="xy")
    n = X.size
    fl = {"x": X.ravel(), "y": Y.ravel(), "u": np.zeros(n), "v": np.zeros(n),
          "p": np.zeros(n), "rho": np.full(n, rho0),
          "m": np.full(n, rho0 * DX * DX), "h": np.full(n, hdx * DX)}
    wy = -(np.arange(layers) + 0.5) * DX
    WX, WY = np.meshgrid(gx, wy, indexing="xy")
    nw = WX.size
    walls = {"x": WX.ravel(), "y": WY.ravel(), "h": np.full(nw, hdx * DX),
             "m": np.full(nw, rho0 * DX * DX)}
    P = oracle.params(lo=(0.0, -1.0), hi=(nx * DX, 1.0), periodic=(1, 0),
                      rho0=rho0, cs=10.0, nu=0.01, hdx=hdx)
    return fl, walls, P


def _rhs(P, fl, walls, dt=1e-4):
    oracle.set_walls(walls)
    try:
        return oracle.rhs(P, dt, oracle.make_state(fl))
    finally:
        oracle.set_walls(None)


def test_shepard_reproduces_constants():
    fl, walls, P = _half_plane()
    fl["p"][:] = 3.5
    fl["u"][:] = 0.7
    fl["v"][:] = -0.2
    walls["u"] = np.full(len(walls["x"]), 0.1)
    oracle.set_walls(walls)
    try:
        bc = oracle.wall_bc(P, oracle.make_state(fl), len(walls["x"]))
    finally:
        oracle.set_walls(None)
    reach = walls["y"] > -3 * DX          # walls with fluid in range
    assert reach.sum() > 0 and (~reach).sum() > 0
    assert np.allclose(bc["p"][reach], 3.5, rtol=1e-14, atol=0)
    assert np.allclose(bc["ugx"][reach], 2 * 0.1 - 0.7, rtol=0, atol=1e-14)
    assert np.allclose(bc["ugy"][reach], 0.2, rtol=0, atol=1e-14)
    # no fluid in range: zero pressure and the plain mirror of 0
    assert np.all(bc["p"][~reach] == 0.0)
    assert np.allclose(bc["ugx"][~reach], 0.2, rtol=0, atol=0)


def test_walls_restore_density_support():
    fl, walls, P = _half_plane()
    with_w = _rhs(P, fl, walls)
    without = oracle.rhs(P, 1e-4, oracle.make_state(fl))
    first = fl["y"] < DX                       # the row next to the wall
    assert np.abs(with_w["rho"][first] - 1.0).max() < 2e-3
    assert without["rho"][first].max() < 0.9


def test_uniform_pressure_at_rest_is_force_free_at_a_wall():
    fl, walls, P = _half_plane()
    fl["p"][:] = 2.0
    r = _rhs(P, fl, walls)
    inner = fl["y"] < 10 * DX                  # away from the open top
    scale = r["s_dvdt"][inner].max()
    assert np.abs(r["dvdt"][inner]).max() < 1e-3 * scale
    assert np.abs(r["dudt"][inner]).max() < 1e-12 * scale
    # the wall pressure enters p_avg: a wrong wall pressure would show as a
    # force on the first rows
    bad = dict(walls)
    oracle.set_walls(bad)
    try:
        st = oracle.make_state(dict(fl, p=np.where(fl["y"] < DX, 2.0, 2.0)))
        r2 = oracle.rhs(P, 1e-4, st)
    finally:
        oracle.set_walls(None)
    assert np.abs(r2["dvdt"][inner]).max() < 1e-3 * scale


def test_wall_moving_with_the_stream_adds_nothing():
    fl, walls, P = _half_plane()
    fl["u"][:] = 0.6
    walls["u"] = np.full(len(walls["x"]), 0.6)
    r = _rhs(P, fl, walls)
    inner = fl["y"] < 10 * DX
    for k in ("dudt", "dvdt", "dpdt"):
        assert np.abs(r[k][inner]).max() <= 1e-12 * max(r["s_" + k].max(), 1)


def test_flow_into_a_wall_compresses():
    fl, walls, P = _half_plane()
    fl["v"][:] = -0.3
    r = _rhs(P, fl, walls)
    first = fl["y"] < DX
    mid = (fl["y"] > 6 * DX) & (fl["y"] < 10 * DX)
    assert r["dpdt"][first].min() > 0.0
    assert np.abs(r["dpdt"][mid]).max() < 1e-9 * r["s_dpdt"][mid].max()
