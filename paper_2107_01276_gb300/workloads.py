"""Seeded synthetic particle sets shaped like the paper's workloads.

This module only lays particles out and draws random numbers; it holds none
of the SPH method's arithmetic, and both the CUDA path and the CPU oracle
take their inputs from it.  Each generator returns a dict with the particle
arrays (FP64 numpy) and a ``params`` dict of physical parameters that both
sides translate into their own parameter blocks.

Workloads (all synthetic; the paper's runs use no external data set):
  taylor_green   -- Taylor-Green vortex on the periodic unit square, the
                    initial condition of section 4.1 (Eq. tgv_sol at t = 0).
  perturbed      -- lattice with position jitter and a smooth h variation,
                    for parity at sizes the oracle finishes in seconds.
  half_plane_walls -- fluid above rows of dummy wall particles (parity of
                    the wall boundary condition).
  cylinder       -- flow past a circular cylinder (section 4.4) with wall
                    rings, a background graded by C_r per ring, and a coarse
                    fluid lattice that sph_adapt refines.
  graded_strip   -- periodic square whose column spacing grows by the
                    paper's layer ratio C_r from a fine core to 1:ratio (the
                    pair-kernel sweep), symmetric so the spacing is
                    continuous across the periodic wrap.
"""
from __future__ import annotations

import math

import numpy as np


def _base_params(**kw):
    p = dict(lo=(0.0, 0.0), hi=(1.0, 1.0), periodic=(1, 1), rho0=1.0,
             cs=10.0, nu=0.0, U_ref=1.0, hdx=1.0, alpha_e=1.5,
             split_alpha=0.9, split_eps=0.4, ds_min=0.0, ds_max=0.0,
             Cr=1.08, pavg_mode=0, edac_diff_denominator=1,
             edac_rho_factor=1, merge_iters=3, shift_iters=3)
    p.update(kw)
    return p


def taylor_green(nx: int = 50, Re: float = 100.0, L: float = 1.0,
                 hdx: float = 1.0, rho0: float = 1.0, cs: float = 10.0,
                 U: float = 1.0, jitter: float = 0.0, seed: int = 1):
    """nx*nx lattice on [0, L)^2, periodic; u, v, p from the Taylor-Green
    closed form at t = 0 (section 4.1), nu = U L / Re."""
    dx = L / nx
    g = (np.arange(nx) + 0.5) * dx
    X, Y = np.meshgrid(g, g, indexing="xy")
    x, y = X.ravel().copy(), Y.ravel().copy()
    if jitter > 0:
        rng = np.random.default_rng(seed)
        x += jitter * dx * rng.uniform(-1, 1, x.size)
        y += jitter * dx * rng.uniform(-1, 1, y.size)
        x %= L
        y %= L
    k = 2.0 * math.pi / L
    u = -U * np.cos(k * x) * np.sin(k * y)
    v = U * np.sin(k * x) * np.cos(k * y)
    p = -rho0 * U * U * (np.cos(2 * k * x) + np.cos(2 * k * y)) / 4.0
    n = x.size
    parts = dict(x=x, y=y, u=u, v=v, p=p, rho=np.full(n, rho0),
                 m=np.full(n, rho0 * dx * dx), h=np.full(n, hdx * dx))
    params = _base_params(lo=(0.0, 0.0), hi=(L, L), periodic=(1, 1),
                          rho0=rho0, cs=cs, nu=U * L / Re, U_ref=U, hdx=hdx)
    return dict(particles=parts, params=params, dx=dx, Re=Re, L=L, U=U)


def _lattice(lo, hi, ds):
    """Cell-centred lattice of spacing ~ds on the box [lo, hi)."""
    nx = max(1, int(round((hi[0] - lo[0]) / ds)))
    ny = max(1, int(round((hi[1] - lo[1]) / ds)))
    gx = lo[0] + (np.arange(nx) + 0.5) * (hi[0] - lo[0]) / nx
    gy = lo[1] + (np.arange(ny) + 0.5) * (hi[1] - lo[1]) / ny
    X, Y = np.meshgrid(gx, gy, indexing="xy")
    return X.ravel().copy(), Y.ravel().copy()


def _background_lattice(lo, hi, ds_max, hdx, rho0):
    """Background particles for the construction of section 3.3: a ds_max
    lattice over the box with h = hdx ds_max and m = rho0 ds_max^2."""
    x, y = _lattice(lo, hi, ds_max)
    n = x.size
    return dict(x=x, y=y, h=np.full(n, hdx * ds_max), ds=np.full(n, ds_max),
                m=np.full(n, rho0 * ds_max * ds_max))


def _markers(lo, hi, ds, hdx, inside):
    """Refinement-region markers (section 3.3, user-specified regions): a
    ds lattice over the box kept where inside(x, y)."""
    x, y = _lattice(lo, hi, ds)
    keep = inside(x, y)
    n = int(keep.sum())
    return dict(x=x[keep], y=y[keep], h=np.full(n, hdx * ds))


def taylor_green_adaptive(nx: int = 50, Re: float = 100.0, L: float = 1.0,
                          hdx: float = 1.0, rho0: float = 1.0,
                          cs: float = 10.0, U: float = 1.0,
                          zone=(0.1, 0.5), ratio: float = 2.0,
                          Cr: float = 1.08):
    """Taylor-Green vortex with an inner refinement zone [0.1 L, 0.5 L]^2 at
    `ratio` times the outer resolution (section 4.1): fluid on the outer
    nx*nx lattice with the closed-form fields, a background lattice at
    ds_max = L/nx to be built by sph_background, and region markers filling
    the zone at ds_min = ds_max / ratio."""
    d = taylor_green(nx=nx, Re=Re, L=L, hdx=hdx, rho0=rho0, cs=cs, U=U)
    ds_max = L / nx
    ds_min = ds_max / ratio
    z0, z1 = zone[0] * L, zone[1] * L
    d["params"].update(ds_min=ds_min, ds_max=ds_max, Cr=Cr)
    d["background"] = _background_lattice((0.0, 0.0), (L, L), ds_max, hdx, rho0)
    d["region"] = _markers((z0, z0), (z1, z1), ds_min, hdx,
                           lambda x, y: np.ones(x.size, bool))
    d["construct_background"] = True
    d["zone"] = (z0, z1)
    return d


def gresho_chan(nx: int = 50, hdx: float = 1.0, rho0: float = 1.0,
                cs: float = 10.0, p0: float = 5.0, R: float = 0.2,
                adaptive: bool = True, r_region: float = 0.45,
                mass_ratio: float = 0.5, Cr: float = 1.08):
    """Gresho-Chan vortex (section 4.2): inviscid, periodic unit box centred
    on the vortex, Cartesian lattice, azimuthal velocity and pressure from
    Eqs. gc-az and gc-p (p0 = 5, R = 0.2 L).  Beyond 2R the pressure is
    p0 + 4 log 2 - 2, the value that keeps p continuous (dp/dr = u^2 / r);
    the printed constant 4 log 2 - 4 would leave a jump of 2 at r = 2R.  Adaptive: region markers fill
    the half disc y >= 0 of radius r_region around the centre at the size
    whose reference mass is mass_ratio times the outer one, and a
    background lattice at ds_max = L / nx is to be built."""
    L = 1.0
    dx = L / nx
    x, y = _lattice((-0.5, -0.5), (0.5, 0.5), dx)
    r = np.hypot(x, y)
    q = r / R
    uphi = np.where(q < 1, q, np.where(q < 2, 2 - q, 0.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        p = np.where(r < R, 12.5 * r * r,
                     np.where(r < 2 * R,
                              4 - 4 * math.log(0.2) + 12.5 * r * r - 20 * r
                              + 4 * np.log(np.maximum(r, 1e-300)),
                              4 * math.log(2.0) - 2))
    p = p0 + p
    rs = np.where(r > 0, r, 1.0)
    u = -uphi * y / rs
    v = uphi * x / rs
    n = x.size
    parts = dict(x=x, y=y, u=u, v=v, p=rho0 * p, rho=np.full(n, rho0),
                 m=np.full(n, rho0 * dx * dx), h=np.full(n, hdx * dx))
    params = _base_params(lo=(-0.5, -0.5), hi=(0.5, 0.5), periodic=(1, 1),
                          rho0=rho0, cs=cs, nu=0.0, U_ref=1.0, hdx=hdx)
    d = dict(particles=parts, params=params, dx=dx, R=R, p0=p0)
    if adaptive:
        ds_max = dx
        ds_min = dx * math.sqrt(mass_ratio)
        params.update(ds_min=ds_min, ds_max=ds_max, Cr=Cr)
        d["background"] = _background_lattice((-0.5, -0.5), (0.5, 0.5),
                                              ds_max, hdx, rho0)
        d["region"] = _markers((-0.5, -0.5), (0.5, 0.5), ds_min, hdx,
                               lambda xx, yy: (np.hypot(xx, yy) < r_region)
                               & (yy >= 0))
        d["construct_background"] = True
    return d


def gresho_chan_exact(x, y, R: float = 0.2):
    """Azimuthal speed of the Gresho-Chan vortex at (x, y) (Eq. gc-az)."""
    q = np.hypot(x, y) / R
    return np.where(q < 1, q, np.where(q < 2, 2 - q, 0.0))


def perturbed(nx: int = 40, ny: int = 32, L: float = 1.0, hdx: float = 1.2,
              h_ratio: float = 2.0, jitter: float = 0.15,
              periodic=(1, 1), rho0: float = 1.0, cs: float = 10.0,
              nu: float = 0.01, seed: int = 3):
    """nx*ny lattice with jitter, random velocities and pressures, and a
    smooth h variation by ``h_ratio`` across x; masses follow h."""
    rng = np.random.default_rng(seed)
    Ly = L * ny / nx
    dx = L / nx
    gx = (np.arange(nx) + 0.5) * dx
    gy = (np.arange(ny) + 0.5) * (Ly / ny)
    X, Y = np.meshgrid(gx, gy, indexing="xy")
    x = X.ravel() + jitter * dx * rng.uniform(-1, 1, X.size)
    y = Y.ravel() + jitter * dx * rng.uniform(-1, 1, X.size)
    if periodic[0]:
        x %= L
    if periodic[1]:
        y %= Ly
    n = x.size
    # spacing varies smoothly (periodic-compatible) by h_ratio
    s = dx * h_ratio ** (0.5 - 0.5 * np.cos(2 * math.pi * x / L))
    s = s / h_ratio ** 0.5
    h = hdx * s
    m = rho0 * s * s
    u = rng.normal(0.0, 0.1, n)
    v = rng.normal(0.0, 0.1, n)
    rho = rho0 * (1.0 + rng.uniform(-0.01, 0.01, n))
    p = rng.normal(0.0, 0.2, n)
    parts = dict(x=x, y=y, u=u, v=v, p=p, rho=rho, m=m, h=h)
    params = _base_params(lo=(0.0, 0.0), hi=(L, Ly), periodic=tuple(periodic),
                          rho0=rho0, cs=cs, nu=nu, U_ref=1.0, hdx=hdx)
    return dict(particles=parts, params=params, dx=dx)


def _graded_columns(d_min, ratio, Cr, L):
    """Column spacings of a symmetric graded strip: spacing d_min in a core
    of 8 columns at x = L/2, growing by Cr per column to ratio*d_min, then
    constant out to both (periodic) ends."""
    d_max = ratio * d_min
    half = [d_min] * 4
    d = d_min
    while d < d_max:
        d = min(d * Cr, d_max)
        half.append(d)
    width = sum(half)
    if width > 0.5 * L:
        raise ValueError("grading does not fit the domain")
    n_out = max(1, int(round((0.5 * L - width) / d_max)))
    half += [d_max] * n_out
    cols = half[::-1] + half            # coarse ... fine fine ... coarse
    x = np.cumsum([0.0] + cols[:-1])
    x = x * (L / sum(cols))
    w = np.array(cols) * (L / sum(cols))
    return x, w


def graded_strip(n_target: int = 1 << 20, ratio: float = 250.0,
                 Cr: float = 1.08, hdx: float = 1.2, rho0: float = 1.0,
                 cs: float = 10.0, nu: float = 0.0, seed: int = 4):
    """Periodic unit square of columns whose spacing grows geometrically,
    by Cr from one column to the next (the paper's layer ratio, section
    3.3), from dx_min in a core at x = L/2 to ratio*dx_min, then stays
    constant to x = 0 and L.  Column k holds round(L/dx_k) particles at
    spacing L/ny_k.  h = hdx*sqrt(dx dy), m = rho0*dx*dy; u, v ~ N(0, 0.1);
    rho = rho0 (1 + U(-0.01, 0.01)); p = rho0 cs^2 (rho/rho0 - 1).  dx_min
    is chosen so the particle count is close to n_target."""
    rng = np.random.default_rng(seed)
    L = 1.0

    def count(dmin):
        try:
            x, w = _graded_columns(dmin, ratio, Cr, L)
        except ValueError:
            return None
        return int(sum(max(1, int(round(L / d))) for d in w))

    lo, hi = 1e-7, 1.0 / (2.0 * ratio)
    while count(hi) is None:
        hi *= 0.7
    for _ in range(60):
        mid = math.sqrt(lo * hi)
        c = count(mid)
        if c is None or c < n_target:
            hi = mid
        else:
            lo = mid
    dx_min = lo if count(lo) is not None else hi
    xs, ws = _graded_columns(dx_min, ratio, Cr, L)
    cx, cy, cdx, cdy = [], [], [], []
    for xc, d in zip(xs, ws):
        ny = max(1, int(round(L / d)))
        dy = L / ny
        cx.append(np.full(ny, xc + 0.5 * d))
        cy.append((np.arange(ny) + 0.5) * dy)
        cdx.append(np.full(ny, d))
        cdy.append(np.full(ny, dy))
    x = np.concatenate(cx) % L
    y = np.concatenate(cy)
    ddx = np.concatenate(cdx)
    ddy = np.concatenate(cdy)
    n = x.size
    s = np.sqrt(ddx * ddy)
    u = rng.normal(0.0, 0.1, n)
    v = rng.normal(0.0, 0.1, n)
    rho = rho0 * (1.0 + rng.uniform(-0.01, 0.01, n))
    p = rho0 * cs * cs * (rho / rho0 - 1.0)
    parts = dict(x=x, y=y, u=u, v=v, p=p, rho=rho, m=rho0 * ddx * ddy,
                 h=hdx * s)
    params = _base_params(lo=(0.0, 0.0), hi=(L, L), periodic=(1, 1),
                          rho0=rho0, cs=cs, nu=nu, U_ref=1.0, hdx=hdx,
                          ds_min=float(s.min()), Cr=Cr)
    return dict(particles=parts, params=params, dx_min=float(s.min()))


def half_plane_walls(nx: int = 30, ny: int = 20, layers: int = 4,
                     dx: float = 0.02, hdx: float = 1.2, rho0: float = 1.0,
                     cs: float = 10.0, nu: float = 0.01, jitter: float = 0.1,
                     seed: int = 21):
    """Fluid lattice y > 0 above `layers` rows of wall particles (y < 0) on
    an x-periodic strip; jittered fluid, random u, v, p."""
    rng = np.random.default_rng(seed)
    gx = (np.arange(nx) + 0.5) * dx
    gy = (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(gx, gy, indexing="xy")
    n = X.size
    x = (X.ravel() + jitter * dx * rng.uniform(-1, 1, n)) % (nx * dx)
    y = Y.ravel() + jitter * dx * rng.uniform(-0.5, 1, n)
    fl = dict(x=x, y=y, u=rng.normal(0, 0.1, n), v=rng.normal(0, 0.1, n),
              p=rng.normal(0, 0.3, n), rho=np.full(n, rho0),
              m=np.full(n, rho0 * dx * dx), h=np.full(n, hdx * dx))
    wy = -(np.arange(layers) + 0.5) * dx
    WX, WY = np.meshgrid(gx, wy, indexing="xy")
    nw = WX.size
    walls = dict(x=WX.ravel(), y=WY.ravel(), h=np.full(nw, hdx * dx),
                 m=np.full(nw, rho0 * dx * dx), u=np.full(nw, 0.05),
                 v=np.zeros(nw))
    params = _base_params(lo=(0.0, -1.0), hi=(nx * dx, 1.0), periodic=(1, 0),
                          rho0=rho0, cs=cs, nu=nu, U_ref=1.0, hdx=hdx)
    return dict(particles=fl, walls=walls, params=params, dx=dx)


def cylinder(D: float = 2.0, Re: float = 40.0, ds_min_over_D: float = 1 / 50,
             ds_max_over_D: float = 0.5, Lx_over_D: float = 25.0,
             Ly_over_D: float = 15.0, center_over_D=(7.5, 7.5),
             rho0: float = 1000.0, cs: float = 10.0, U: float = 1.0,
             hdx: float = 1.2, Cr: float = 1.08, jitter: float = 1e-3,
             wall_layers: int = 4, seed: int = 2,
             background: str = "construct", fluid: str = "lattice"):
    """Flow past a circular cylinder (section 4.4, Table fpc-params: D = 2,
    rho0 = 1000, c_s = 10, h/dx = 1.2, C_r = 1.08), periodic box of
    25D x 15D, impulsive start u = U.

    - walls: `wall_layers` rings of dummy particles inside the cylinder at
      spacing ds_min (section 2.2);
    - background, `background="construct"` (default): a ds_max lattice
      over the whole box (h = hdx ds_max, m = rho0 ds_max^2) to be refined
      by the construction of section 3.3 (sph_background) before use; the
      dict then has construct_background = True.  `background="rings"`:
      rings around the cylinder whose size grows by C_r per ring from
      ds_min at the wall to ds_max, then a ds_max lattice -- the graded
      layers the construction aims at, given directly;
    - background_rings: the ring background in either case;
    - fluid, `fluid="lattice"` (default): a ds_max lattice outside the
      cylinder with 1e-3 ds_max position jitter; sph_adapt refines it to
      the background's sizes.  `fluid="rings"`: one fluid particle at each
      ring-background particle (m = rho0 ds^2, h = hdx ds, 1e-3 ds jitter),
      the fluid initialised from the background particles (section 3.4,
      step 2; for large spacing ratios, where refining a ds_max lattice by
      splitting piles 7^k children into clusters that shifting cannot
      spread).
    """
    rng = np.random.default_rng(seed)
    R = 0.5 * D
    cx, cy = center_over_D[0] * D, center_over_D[1] * D
    Lx, Ly = Lx_over_D * D, Ly_over_D * D
    ds_min, ds_max = ds_min_over_D * D, ds_max_over_D * D
    # walls
    wx, wy = [], []
    for k in range(wall_layers):
        r = R - (k + 0.5) * ds_min
        nk = max(3, int(round(2 * math.pi * r / ds_min)))
        th = (np.arange(nk) + 0.5 * (k % 2)) * 2 * math.pi / nk
        wx.append(cx + r * np.cos(th))
        wy.append(cy + r * np.sin(th))
    wx, wy = np.concatenate(wx), np.concatenate(wy)
    nw = wx.size
    walls = dict(x=wx, y=wy, h=np.full(nw, hdx * ds_min),
                 m=np.full(nw, rho0 * ds_min * ds_min), u=np.zeros(nw),
                 v=np.zeros(nw))
    # background rings, sizes growing by Cr per ring
    bx, by, bds = [], [], []
    r, ds = R + 0.5 * ds_min, ds_min
    while ds < ds_max:
        nk = max(6, int(round(2 * math.pi * r / ds)))
        th = np.arange(nk) * 2 * math.pi / nk
        bx.append(cx + r * np.cos(th))
        by.append(cy + r * np.sin(th))
        bds.append(np.full(nk, ds))
        r += ds
        ds = min(ds * Cr, ds_max)
    r_ring = r
    gxs = (np.arange(int(round(Lx / ds_max))) + 0.5) * ds_max
    gys = (np.arange(int(round(Ly / ds_max))) + 0.5) * ds_max
    GX, GY = np.meshgrid(gxs, gys, indexing="xy")
    far = np.hypot(GX - cx, GY - cy) >= r_ring
    bx.append(GX[far])
    by.append(GY[far])
    bds.append(np.full(int(far.sum()), ds_max))
    rings = dict(x=np.concatenate(bx) % Lx, y=np.concatenate(by) % Ly,
                 ds=np.concatenate(bds))
    rings["h"] = hdx * rings["ds"]
    nb = GX.size
    lattice = dict(x=GX.ravel().copy(), y=GY.ravel().copy(),
                   h=np.full(nb, hdx * ds_max), ds=np.full(nb, ds_max),
                   m=np.full(nb, rho0 * ds_max * ds_max))
    # fluid: coarse lattice outside the cylinder
    inside = np.hypot(GX - cx, GY - cy) < R + 0.5 * ds_max
    fx, fy = GX[~inside].ravel(), GY[~inside].ravel()
    n = fx.size
    fx = (fx + jitter * ds_max * rng.uniform(-1, 1, n)) % Lx
    fy = (fy + jitter * ds_max * rng.uniform(-1, 1, n)) % Ly
    fl = dict(x=fx, y=fy, u=np.full(n, U), v=np.zeros(n), p=np.zeros(n),
              rho=np.full(n, rho0), m=np.full(n, rho0 * ds_max * ds_max),
              h=np.full(n, hdx * ds_max))
    if fluid == "rings":
        keep = np.hypot(rings["x"] - cx, rings["y"] - cy) >= R
        ds = rings["ds"][keep]
        n = int(keep.sum())
        fx = (rings["x"][keep] + jitter * ds * rng.uniform(-1, 1, n)) % Lx
        fy = (rings["y"][keep] + jitter * ds * rng.uniform(-1, 1, n)) % Ly
        fl = dict(x=fx, y=fy, u=np.full(n, U), v=np.zeros(n), p=np.zeros(n),
                  rho=np.full(n, rho0), m=rho0 * ds * ds, h=hdx * ds)
    elif fluid != "lattice":
        raise ValueError("fluid must be 'lattice' or 'rings'")
    params = _base_params(lo=(0.0, 0.0), hi=(Lx, Ly), periodic=(1, 1),
                          rho0=rho0, cs=cs, nu=U * D / Re, U_ref=U, hdx=hdx,
                          ds_min=ds_min, ds_max=ds_max, Cr=Cr)
    if background not in ("construct", "rings"):
        raise ValueError("background must be 'construct' or 'rings'")
    out = dict(particles=fl, walls=walls, params=params, D=D, Re=Re, U=U,
               background_rings=rings)
    if background == "construct":
        out["background"] = lattice
        out["construct_background"] = True
    else:
        out["background"] = rings
    return out


def subset(parts: dict, idx) -> dict:
    return {k: np.asarray(v)[idx].copy() for k, v in parts.items()}


def ring_in_lattice(ds: float = 0.05, R: float = 1.0, box: float = 6.0,
                    layers: int = 4, hdx: float = 1.2, rho0: float = 1.0,
                    cs: float = 10.0, nu: float = 0.01, jitter: float = 0.0,
                    seed: int = 1):
    """A closed circular body of radius R at the centre of a periodic
    box x box: `layers` rings of wall particles at spacing ds inside r < R,
    fluid on the ds lattice outside (optionally jittered), at rest with
    zero pressure (callers set the fields).  Returns particles, walls,
    params and the centre."""
    rng = np.random.default_rng(seed)
    g = (np.arange(int(round(box / ds))) + 0.5) * ds
    X, Y = np.meshgrid(g, g, indexing="xy")
    x, y = X.ravel(), Y.ravel()
    c = 0.5 * box
    keep = np.hypot(x - c, y - c) >= R
    x, y = x[keep], y[keep]
    if jitter > 0:
        x = x + jitter * ds * rng.uniform(-1, 1, x.size)
        y = y + jitter * ds * rng.uniform(-1, 1, y.size)
    n = x.size
    fl = dict(x=x, y=y, u=np.zeros(n), v=np.zeros(n), p=np.zeros(n),
              rho=np.full(n, rho0), m=np.full(n, rho0 * ds * ds),
              h=np.full(n, hdx * ds))
    wx, wy = [], []
    for k in range(layers):
        r = R - (k + 0.5) * ds
        nk = 2 * int(round(math.pi * r / ds))   # even: mirror-symmetric
        t = (np.arange(nk) + 0.5) * (2 * math.pi / nk)
        wx.append(c + r * np.cos(t))
        wy.append(c + r * np.sin(t))
    wx, wy = np.concatenate(wx), np.concatenate(wy)
    walls = dict(x=wx, y=wy, h=np.full(wx.size, hdx * ds),
                 m=np.full(wx.size, rho0 * ds * ds))
    params = _base_params(lo=(0.0, 0.0), hi=(box, box), periodic=(1, 1),
                          rho0=rho0, cs=cs, nu=nu, U_ref=1.0, hdx=hdx)
    return {"particles": fl, "walls": walls, "params": params,
            "center": (c, c), "R": R, "ds": ds}
