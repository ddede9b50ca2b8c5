"""User-specified refinement regions (section 3.3) and the two workloads of
section 4 that use them, on the GPU: the Taylor-Green vortex with a
refined inner square (section 4.1) and the adaptive Gresho-Chan vortex
(section 4.2).

Parity with the oracle (inputs from the generators or the oracle itself):
one background iteration with region markers, the full background
construction's particle count, one adaptation against the oracle's own
background, and the right-hand side of the Gresho-Chan fields.  Validation
against the closed forms: the adaptive Taylor-Green vortex decays as
exp(-8 pi^2 t / Re) and the adaptive Gresho-Chan vortex keeps its velocity
profile, both with mass conserved to rounding."""
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


def _sim(d, precision=sph.SPH_FP64, cap=200000, background=None):
    P = sph.make_params(d["params"], precision=precision, capacity=cap,
                        bg_capacity=200000)
    s = sph.Simulation(P, stream_handle())
    s.load(d["particles"])
    if "region" in d:
        s.load(d["region"], kind=sph.SPH_REGION)
    bg = background if background is not None else d.get("background")
    if bg is not None:
        s.load(bg, kind=sph.SPH_BACKGROUND)
    return s


@pytest.fixture(scope="module")
def tgv_oracle_background():
    """The oracle's construction for the adaptive Taylor-Green vortex (region
    markers as the solid): its state after 2 iterations and at the end."""
    d = wl.taylor_green_adaptive(nx=50)
    pr = d["params"]
    P = oracle.params(**pr)
    B = oracle.bg_params(pr["ds_min"], pr["ds_max"], pr["Cr"])
    b = oracle.make_bgset(d["background"], cap=100000)
    nid = b["n"]
    stage2 = None
    for it in range(oracle.bg_iterations(B)):
        if it == 2:
            stage2 = {k: b[k][:b["n"]].copy() for k in oracle.BG_FIELDS + ("id",)}
        r, _, nid = oracle.bg_iteration(P, B, b, nid, d["region"])
        assert r == 0
    final = {k: b[k][:b["n"]].copy() for k in oracle.BG_FIELDS + ("id",)}
    return d, stage2, final


def test_region_marking_iteration_parity(tgv_oracle_background):
    d, stage2, _ = tgv_oracle_background
    s = _sim(d, background=stage2)
    g = s.background(1)
    got = s.read_background()
    s.close()
    order = np.argsort(got["id"])
    got = {k: v[order] for k, v in got.items()}
    pr = d["params"]
    P = oracle.params(**pr)
    B = oracle.bg_params(pr["ds_min"], pr["ds_max"], pr["Cr"])
    b = oracle.make_bgset(stage2, cap=100000)
    r, o, _ = oracle.bg_iteration(P, B, b, int(stage2["id"].max()) + 1,
                                  d["region"])
    assert r == 0 and o["n_marked"] > 0
    for k in ("n_marked", "n_split", "n_after"):
        assert g[k] == o[k], k
    n = b["n"]
    ro = np.argsort(b["id"][:n])
    assert np.array_equal(got["id"], b["id"][:n][ro])
    assert np.array_equal(got["m"], b["m"][:n][ro])
    assert np.abs(got["ds"] / b["ds"][:n][ro] - 1).max() < 1e-12
    assert np.abs(got["h"] / b["h"][:n][ro] - 1).max() < 1e-12


def test_region_construction_count_matches_oracle(tgv_oracle_background):
    d, _, final = tgv_oracle_background
    s = _sim(d)
    g = s.background()
    assert g["iterations"] == 30
    n = s.info()["n_bg"]
    s.close()
    assert abs(n - len(final["x"])) <= 0.01 * len(final["x"])


def test_adaptation_with_the_oracle_background(tgv_oracle_background):
    """One sph_adapt from the Taylor-Green lattice against the oracle's
    constructed background: counts, ids and masses equal the oracle's."""
    d, _, final = tgv_oracle_background
    s = _sim(d, background=final)
    g = s.adapt()
    got = by_id(s, ["m", "mmax"])
    s.close()
    P = oracle.params(**d["params"])
    st = oracle.make_state(d["particles"], cap=200000)
    r, o, _ = oracle.adapt(P, st, bg=final)
    assert r == 0
    assert (g["n_split"], g["n_merged"], g["n_after"]) == \
        (o["n_split"], o["n_merged"], o["n_after"])
    n = st["n"]
    order = np.argsort(st["id"][:n])
    assert np.array_equal(got["id"], st["id"][:n][order])
    assert np.array_equal(got["m"], st["m"][:n][order])
    assert np.array_equal(got["mmax"], st["mmax"][:n][order])


@pytest.mark.parametrize("precision,tol", [(sph.SPH_FP64, FP64_TOL),
                                           (sph.SPH_MIXED, MIXED_TOL)])
def test_gresho_chan_rhs_parity(precision, tol):
    d = wl.gresho_chan(nx=60, adaptive=False)
    s = _sim(d, precision=precision, cap=len(d["particles"]["x"]))
    s.rhs()
    got = by_id(s, list(RHS_FIELDS) + ["nnb"])
    s.close()
    P = oracle.params(**d["params"])
    pt = d["particles"]
    ref = oracle.rhs(P, oracle.dt(P, pt["h"]), oracle.make_state(pt))
    assert np.array_equal(got["nnb"], ref["nnb"])
    for f in RHS_FIELDS:
        assert norm(got[f], ref[f], ref["s_" + f]) <= tol, f


@pytest.mark.parametrize("precision", [sph.SPH_FP64, sph.SPH_MIXED])
def test_adaptive_taylor_green_decays_like_the_closed_form(precision):
    d = wl.taylor_green_adaptive(nx=50)
    s = _sim(d, precision=precision)
    s.background()
    m0 = math.fsum(s.read("m"))
    for _ in range(6):
        s.adapt()
    x, y, m = s.read("x"), s.read("y"), s.read("m")
    z0, z1 = d["zone"]
    inner = (x > z0 + 0.05) & (x < z1 - 0.05) & (y > z0 + 0.05) & (y < z1 - 0.05)
    ds_min = d["params"]["ds_min"]
    assert inner.sum() > 500
    assert m[inner].max() <= 1.05 * ds_min * ds_min       # refined inside
    b = -8 * math.pi ** 2 / d["Re"]
    u0 = None
    for it in range(40):
        s.adapt()
        t = s.step(5)
        u = np.hypot(s.read("u"), s.read("v")).max()
        if u0 is None:
            u0 = u / math.exp(b * t)
        assert abs(u / (u0 * math.exp(b * t)) - 1) < 1e-2, (it, t)
    assert abs(math.fsum(s.read("m")) - m0) <= 1e-13 * m0
    s.close()


@pytest.mark.parametrize("precision", [sph.SPH_FP64, sph.SPH_MIXED])
def test_adaptive_gresho_chan_keeps_the_vortex(precision):
    d = wl.gresho_chan(nx=50)
    s = _sim(d, precision=precision)
    s.background()
    m0 = math.fsum(s.read("m"))
    for _ in range(4):
        s.adapt()
    x, y, m = s.read("x"), s.read("y"), s.read("m")
    half = (np.hypot(x, y) < 0.35) & (y > 0.05)
    m_outer = d["dx"] ** 2
    assert m[half].max() <= 1.05 * 0.5 * m_outer          # refined half disc

    def l1():
        x, y, u, v = s.read("x"), s.read("y"), s.read("u"), s.read("v")
        return np.abs(np.hypot(u, v) - wl.gresho_chan_exact(x, y)).mean()

    assert l1() < 1e-2
    for _ in range(40):
        s.adapt()
        s.step(5)
    assert l1() < 1e-2
    assert abs(math.fsum(s.read("m")) - m0) <= 1e-13 * m0
    s.close()
