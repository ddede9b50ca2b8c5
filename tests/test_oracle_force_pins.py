"""Pins of the oracle's force on the solid (section "Force computation",
Eq. force-sph, reading F1: pressures without the average offset) against
what mechanics fixes, independent of the formula's own code:

- skin friction of a linear shear u = gamma y over a flat wall equals
  rho0 nu gamma per unit wall length;
- a flat wall under a resting layer carries the pressure at its surface;
- a closed body in a linear pressure field feels -grad p times its area
  (Archimedes), and nothing in a uniform one;
- the viscous force is the reaction of the walls' viscous terms in the
  fluid's momentum rates (up to the fluid's beta_j and eta_j in place of
  the wall's);
- rotating the whole state by 90 degrees rotates the force."""
import math

import numpy as np

import oracle
from paper_2107_01276_gb300 import workloads as wl
from tests.test_oracle_wall_pins import DX, _half_plane


def _forces(P, fl, walls):
    oracle.set_walls(walls)
    try:
        return oracle.forces(P, oracle.make_state(fl))
    finally:
        oracle.set_walls(None)


def test_shear_skin_friction():
    """tau = rho0 nu du/dy on the wall; the SPH sum's boundary error (the
    wall velocity is extrapolated over a kernel support) stays within 3 %."""
    fl, walls, P = _half_plane(nx=40, ny=24)
    gamma = 2.0
    fl["u"][:] = gamma * fl["y"]
    f = _forces(P, fl, walls)
    L = 40 * DX
    tau = 1.0 * 0.01 * gamma
    assert abs(f["fv"][0] / (tau * L) - 1) < 0.03
    assert abs(f["fv"][1]) < 1e-12 * tau * L
    assert np.all(f["fp"] == 0.0)             # p = 0 everywhere


def test_flat_wall_carries_the_surface_pressure():
    """Uniform p0 above a flat wall: force -p0 L (into the wall) to the
    kernel's boundary error; a resting layer p = p0 + G (H - y): the wall
    pressure is extrapolated from the fluid within 3h of it, so the load
    is -p(0) L within 3 h G L."""
    fl, walls, P = _half_plane(nx=40, ny=24)
    L = 40 * DX
    fl["p"][:] = 5.0
    f = _forces(P, fl, walls)
    assert abs(f["fp"][1] / (-5.0 * L) - 1) < 0.01
    assert abs(f["fp"][0]) < 1e-12 * 5.0 * L
    H, G = 24 * DX, 3.0
    fl["p"][:] = 5.0 + G * (H - fl["y"])
    f = _forces(P, fl, walls)
    h = 1.2 * DX
    assert abs(f["fp"][1] + (5.0 + G * H) * L) < 3 * h * G * L


def test_archimedes_on_a_closed_body():
    """p = p0 + G (x - xc) around a disc of radius R: force -G pi R^2 along
    x, to the lattice's staircase of the circle (within 5 % at R / ds = 20);
    uniform pressure: no force (the ring is symmetric)."""
    d = wl.ring_in_lattice(ds=0.05)
    fl, walls = d["particles"], d["walls"]
    P = oracle.params(**d["params"])
    xc = d["center"][0]
    G = 2.0
    fl["p"][:] = 3.0 + G * (fl["x"] - xc)
    f = _forces(P, fl, walls)
    A = math.pi * d["R"] ** 2
    assert abs(f["fp"][0] / (-G * A) - 1) < 0.05
    assert abs(f["fp"][1]) < 1e-10 * G * A
    fl["p"][:] = 3.0
    f = _forces(P, fl, walls)
    assert np.abs(f["fp"]).max() < 1e-10 * 3.0 * 2 * math.pi * d["R"]


def test_viscous_force_is_the_reaction_of_the_fluid():
    """The fluid's momentum rates carry the walls' viscous terms divided by
    the fluid particle's beta_j, with eta_j = 0.001 h_j^2; the force on the
    solid uses beta_w = 1 and eta_w, equal to eta_j here (one h).  With
    beta_j multiplied back, the two are equal and opposite to rounding."""
    d = wl.ring_in_lattice(ds=0.05, jitter=0.2, seed=3)
    fl, walls = d["particles"], d["walls"]
    rng = np.random.default_rng(4)
    n = fl["x"].size
    fl["u"][:] = 1.0 + rng.normal(0, 0.1, n)
    fl["v"][:] = rng.normal(0, 0.1, n)
    fl["p"][:] = rng.normal(0, 0.5, n)
    P = oracle.params(**d["params"])
    oracle.set_walls(walls)
    try:
        st = oracle.make_state(fl)
        f = oracle.forces(P, st)
        out, acc = oracle.rhs_wall_terms(P, 1e-4, st)
    finally:
        oracle.set_walls(None)
    w = fl["m"] * out["beta"]
    react = -(w[:, None] * acc[:, 2:]).sum(0)
    assert np.linalg.norm(f["fv"] - react) < 1e-11 * np.linalg.norm(react)
    # flow along +x past a body at rest drags it along +x
    assert f["fv"][0] > 0


def test_rotation_covariance():
    """Rotating positions and velocities by 90 degrees about the centre of
    the square box rotates both force parts: (fx, fy) -> (-fy, fx)."""
    d = wl.ring_in_lattice(ds=0.05, jitter=0.2, seed=5)
    fl, walls = d["particles"], d["walls"]
    rng = np.random.default_rng(6)
    n = fl["x"].size
    fl["u"][:] = rng.normal(0, 0.3, n)
    fl["v"][:] = rng.normal(0, 0.3, n)
    fl["p"][:] = rng.normal(0, 0.5, n)
    P = oracle.params(**d["params"])
    f0 = _forces(P, fl, walls)
    c = d["center"][0]

    def rot(a):
        r = dict(a)
        r["x"], r["y"] = c - (a["y"] - c), c + (a["x"] - c)
        if "u" in a:
            r["u"], r["v"] = -a["v"], a["u"]
        return r

    f1 = _forces(P, rot(fl), rot(walls))
    for k in ("fp", "fv"):
        s = np.linalg.norm(f0[k]) + 1e-300
        assert abs(f1[k][0] + f0[k][1]) < 1e-9 * s, k
        assert abs(f1[k][1] - f0[k][0]) < 1e-9 * s, k
