"""Parity of sph_adapt (background resolution, split, merge rounds, shift
rounds, h update) with the CPU oracle on identical inputs."""
import math

import numpy as np
import pytest

import oracle
from paper_2107_01276_gb300 import sph
from paper_2107_01276_gb300 import workloads as wl
from tests.helpers import by_id, cuda_ok, stream_handle

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "u", "v", "p", "rho", "m", "h", "mmin", "mmax")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not cuda_ok():
        pytest.skip("no CUDA device")


def _refine_case(nx=30, seed=12, periodic=(1, 1), bgn=60):
    d = wl.perturbed(nx=nx, ny=nx, h_ratio=1.0, jitter=0.1, hdx=1.2,
                     periodic=periodic, seed=seed)
    dx = d["dx"]
    g = (np.arange(bgn) + 0.5) / bgn
    X, Y = np.meshgrid(g, g, indexing="xy")
    bg = {"x": X.ravel(), "y": Y.ravel(), "h": np.full(X.size, 1.2 / bgn)}
    bg["ds"] = np.where(bg["x"] < 0.5, 0.5 * dx, dx)
    return d, bg


def _run_both(d, bg, precision=sph.SPH_FP64, calls=1, cap=20000, **over):
    pr = dict(d["params"], **over)
    P = sph.make_params(pr, precision=precision, capacity=cap)
    sim = sph.Simulation(P, stream_handle())
    sim.load(d["particles"])
    if bg is not None:
        sim.load(bg, kind=sph.SPH_BACKGROUND)
    gst = [sim.adapt() for _ in range(calls)]
    OP = oracle.params(**pr)
    st = oracle.make_state(d["particles"], cap=cap)
    nid = None
    ost = []
    for _ in range(calls):
        r, s, nid = oracle.adapt(OP, st, bg=bg, next_id=nid)
        assert r == 0
        ost.append(s)
    n = st["n"]
    order = np.argsort(st["id"][:n])
    ref = {k: st[k][:n][order] for k in FIELDS}
    ref["id"] = st["id"][:n][order]
    got = by_id(sim, list(FIELDS))
    return sim, gst, ost, got, ref


@pytest.mark.parametrize("precision", [sph.SPH_FP64, sph.SPH_MIXED])
@pytest.mark.parametrize("rounds", [3, 5])
def test_merge_cascade_bit_exact_without_shift(rounds, precision):
    """A lattice four times finer than its background (m_ref = 16 m): every
    round merges, and particles merged in one round merge again in the
    next.  The library runs later rounds on the lists of an earlier build
    while the merged particles stay within their reach and rebuilds when
    they leave it; counts, ids, positions and masses must equal the
    oracle's, which rebuilds before every round."""
    d = wl.perturbed(nx=48, ny=48, h_ratio=1.0, jitter=0.1, hdx=1.2, seed=21)
    dx = d["dx"]
    bgn = 12
    g = (np.arange(bgn) + 0.5) / bgn
    X, Y = np.meshgrid(g, g, indexing="xy")
    bg = {"x": X.ravel(), "y": Y.ravel(), "h": np.full(X.size, 1.2 / bgn),
          "ds": np.full(X.size, 4.0 * dx)}
    sim, gst, ost, got, ref = _run_both(d, bg, precision=precision,
                                        shift_iters=0, merge_iters=rounds)
    assert ost[0]["n_merged"] > d["particles"]["x"].size // 2
    for k in ("n_before", "n_split", "n_merged", "n_after"):
        assert gst[0][k] == ost[0][k], (k, gst[0], ost[0])
    assert np.array_equal(got["id"], ref["id"])
    for k in ("x", "y", "m", "mmin", "mmax", "u", "v", "p"):
        assert np.array_equal(got[k], ref[k]), k
    tol = 1e-13 if precision == sph.SPH_FP64 else 2e-5
    assert np.abs(got["h"] / ref["h"] - 1).max() < tol
    sim.close()


def test_split_merge_bit_exact_without_shift():
    """With no shift rounds every position, mass and bound comes from the
    same FP64 expressions on both sides: identical after split + merges."""
    d, bg = _refine_case()
    sim, gst, ost, got, ref = _run_both(d, bg, shift_iters=0)
    for a, b in zip(gst, ost):
        for k in ("n_before", "n_split", "n_merged", "n_after"):
            assert a[k] == b[k], (k, a, b)
    assert np.array_equal(got["id"], ref["id"])
    for k in ("x", "y", "m", "mmin", "mmax", "u", "v", "p"):
        assert np.array_equal(got[k], ref[k]), k
    # h and rho come from neighbour sums (order may differ)
    assert np.abs(got["h"] / ref["h"] - 1).max() < 1e-13
    assert np.abs(got["rho"] / ref["rho"] - 1).max() < 1e-13
    sim.close()


@pytest.mark.parametrize("precision,tol", [(sph.SPH_FP64, 1e-11),
                                           (sph.SPH_MIXED, 2e-5)])
def test_full_adapt_parity(precision, tol):
    """Whole adaptation (3 merge and 3 shift rounds): counts equal, ids
    equal, masses exact (split and merge decisions are FP64 on both paths);
    positions, h, u, v, p within sum-order rounding (FP64) or the FP32
    shift and density sums of the mixed path."""
    d, bg = _refine_case(seed=13)
    sim, gst, ost, got, ref = _run_both(d, bg, precision=precision)
    for k in ("n_split", "n_merged", "n_after"):
        assert gst[0][k] == ost[0][k], k
    assert np.array_equal(got["id"], ref["id"])
    for k in ("m", "mmin", "mmax"):
        assert np.array_equal(got[k], ref[k]), k
    h = ref["h"]
    for k in ("x", "y"):
        dd = got[k] - ref[k]
        dd -= np.round(dd)                   # periodic unit box
        assert np.abs(dd / h).max() < tol, k
    assert np.abs(got["h"] / h - 1).max() < tol
    for k in ("u", "v", "p"):
        sc = max(np.abs(ref[k]).max(), 1e-30)
        assert np.abs(got[k] - ref[k]).max() < tol * sc, k
    m0 = gst[0]["mass_before"]
    assert abs(gst[0]["mass_after"] - m0) <= 1e-13 * m0
    assert abs(math.fsum(got["m"]) - math.fsum(d["particles"]["m"])) <= \
        1e-14 * m0
    sim.close()


def test_nearest_background_fallback_and_open_box():
    """Background too sparse to be in range of some fluid particles: they
    take the nearest background particle's size; non-periodic box."""
    d, bg = _refine_case(nx=24, seed=5, periodic=(0, 0), bgn=6)
    bg["h"] = np.full(bg["x"].size, 0.01)           # tiny supports
    sim, gst, ost, got, ref = _run_both(d, bg, shift_iters=0, merge_iters=1)
    assert np.array_equal(got["mmax"], ref["mmax"])
    assert gst[0]["n_after"] == ost[0]["n_after"]
    sim.close()


def test_repeated_adaptation_then_steps():
    """Three adaptation calls: the oracle runs its own sequence, and each of
    its states before a call is loaded into a fresh context for one
    sph_adapt call: counts, ids and masses equal.  Then the GPU's own three
    calls followed by PEC steps: the state stays finite and mass is
    conserved."""
    d, bg = _refine_case(seed=14)
    pr = dict(d["params"])
    P = sph.make_params(pr, precision=sph.SPH_FP64, capacity=20000)
    OP = oracle.params(**pr)
    st = oracle.make_state(d["particles"], cap=20000)
    nid = len(d["particles"]["x"])
    for call in range(3):
        n = st["n"]
        before = {k: st[k][:n].copy() for k in FIELDS}
        before["id"] = st["id"][:n].copy()
        sim = sph.Simulation(P, stream_handle())
        sim.load(before)
        sim.load(bg, kind=sph.SPH_BACKGROUND)
        g = sim.adapt()
        after = by_id(sim, ["m"])
        sim.close()
        assert nid == int(before["id"].max()) + 1
        r, o, nid = oracle.adapt(OP, st, bg=bg, next_id=nid)
        assert (g["n_split"], g["n_merged"], g["n_after"]) == \
            (o["n_split"], o["n_merged"], o["n_after"]), call
        n = st["n"]
        order = np.argsort(st["id"][:n])
        assert np.array_equal(after["id"], st["id"][:n][order])
        assert np.array_equal(after["m"], st["m"][:n][order])
    sim = sph.Simulation(P, stream_handle())
    sim.load(d["particles"])
    sim.load(bg, kind=sph.SPH_BACKGROUND)
    for _ in range(3):
        sim.adapt()
    sim.step(5)
    for k in ("x", "y", "u", "v", "p"):
        assert np.all(np.isfinite(sim.read(k)))
    m0 = math.fsum(d["particles"]["m"])
    assert abs(math.fsum(sim.read("m")) - m0) <= 1e-13 * m0
    sim.close()


def test_adapt_capacity_and_state_errors():
    d, bg = _refine_case(nx=20)
    n = len(d["particles"]["x"])
    P = sph.make_params(d["params"], capacity=n + 10)
    sim = sph.Simulation(P, stream_handle())
    with pytest.raises(sph.SphError) as e:
        sim.adapt()
    assert e.value.status == sph.SPH_ESTATE
    sim.load(d["particles"])
    sim.load(bg, kind=sph.SPH_BACKGROUND)
    with pytest.raises(sph.SphError) as e:
        sim.adapt()
    assert e.value.status == sph.SPH_ECAPACITY
    assert len(sim.read("x")) == n
    sim.close()
