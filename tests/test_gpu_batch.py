"""Batched stepping (sph_batch_step): uneven instances of both precisions,
with and without walls, advance together, every per-particle phase as one
persistent launch over all of them, launch by launch or replayed as a
captured graph; each instance reaches exactly the state that sph_step
reaches on it alone.  Argument errors change nothing."""
import gc

import numpy as np
import pytest
import torch

import oracle
from paper_2107_01276_gb300 import sph
from paper_2107_01276_gb300 import workloads as wl
from tests.helpers import by_id, cuda_ok

pytestmark = pytest.mark.gpu
FIELDS = ["x", "y", "u", "v", "p", "rho", "h", "m"]


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not cuda_ok():
        pytest.skip("no CUDA device")


@pytest.fixture(autouse=True)
def _collect():
    gc.collect()


def _cases():
    """Uneven instances: sizes from 2.5k to 25k particles (team sizes 32,
    16 and 4), graded h, walls, both precisions."""
    tg = wl.taylor_green(nx=50)
    pert = wl.perturbed(nx=160, ny=150, h_ratio=3.0, seed=5)
    walls = wl.half_plane_walls(nx=60, ny=40, seed=8)
    ring = wl.ring_in_lattice(ds=0.05, jitter=0.1, seed=9)
    rng = np.random.default_rng(10)
    ring["particles"]["u"][:] = 0.5 + rng.normal(0, 0.05, ring["particles"]["x"].size)
    return [(tg, sph.SPH_MIXED), (pert, sph.SPH_MIXED), (walls, sph.SPH_MIXED),
            (ring, sph.SPH_MIXED), (tg, sph.SPH_FP64), (walls, sph.SPH_FP64)]


def _make(d, precision, stream, team=0):
    n = len(d["particles"]["x"])
    P = sph.make_params(d["params"], precision=precision, capacity=n)
    s = sph.Simulation(P, stream)
    if team:
        s.set_tuning(team_a=team, team_b=team)
    s.load(d["particles"])
    if "walls" in d:
        s.load(d["walls"], kind=sph.SPH_WALL)
    return s


@pytest.mark.parametrize("graphs", [False, True])
def test_batch_equals_alone(graphs):
    """Pass A / B team sizes set on the contexts: the batch keeps them (its
    build's walk team follows the batch, which changes no list), so every
    result is bit for bit that of the context alone."""
    cases = _cases()
    steps = 7
    bs = torch.cuda.Stream()
    own = [torch.cuda.Stream() for _ in cases]
    alone = [_make(d, p, st.cuda_stream, 4) for (d, p), st in zip(cases, own)]
    mixed = [_make(d, p, st.cuda_stream, 4) for (d, p), st in zip(cases, own)]
    ta = None
    for _ in range(steps):
        ta = [s.step(1) for s in alone]
    with sph.Batch(len(cases), bs.cuda_stream) as b:
        b.set_graphs(graphs)
        tb = None
        for _ in range(steps):
            tb = b.step(mixed, want_time=True)
        assert b.launches > 0
        # captured at the third call, replayed after (two graphs alternate)
        assert b.graph_steps == (steps - 2 if graphs else 0)
    for q, (a, m) in enumerate(zip(alone, mixed)):
        assert ta[q] == tb[q], q
        ra, rm = by_id(a, FIELDS), by_id(m, FIELDS)
        assert np.array_equal(ra["id"], rm["id"]), q
        for f in FIELDS:
            assert np.array_equal(ra[f], rm[f]), (q, f)
        assert m.info()["steps"] == steps
    for s in alone + mixed:
        s.close()


def test_batch_teams_by_total_size():
    """Untuned contexts: the batch picks pass A / B teams for its total
    particle count; the states differ from the contexts' own runs by the
    order of the pair sums only (rounding)."""
    cases = _cases()
    steps = 4
    bs = torch.cuda.Stream()
    own = [torch.cuda.Stream() for _ in cases]
    alone = [_make(d, p, st.cuda_stream) for (d, p), st in zip(cases, own)]
    mixed = [_make(d, p, st.cuda_stream) for (d, p), st in zip(cases, own)]
    for _ in range(steps):
        for s in alone:
            s.step(1)
    with sph.Batch(len(cases), bs.cuda_stream) as b:
        for _ in range(steps):
            b.step(mixed, want_time=True)
    for q, ((d, prec), a, m) in enumerate(zip(cases, alone, mixed)):
        ra, rm = by_id(a, FIELDS), by_id(m, FIELDS)
        # FP32 pair sums in another order: rates differ by a few 1e-7 of
        # the sums of their terms, which exceed the rates many times where
        # pressure terms cancel; four steps carry that into u, v, p, x, y
        rtol = 1e-11 if prec == sph.SPH_FP64 else 1e-4
        for f in ("u", "v", "p"):
            scale = max(np.max(np.abs(ra[f])), 1e-30)
            assert np.max(np.abs(ra[f] - rm[f])) <= rtol * scale, (q, f)
        dx = np.min(d["particles"]["h"]) / 1.2
        for f in ("x", "y"):
            assert np.max(np.abs(ra[f] - rm[f])) <= rtol * dx, (q, f)
    for s in alone + mixed:
        s.close()


def test_one_launch_per_phase_whatever_the_count():
    """Small instances of one precision and team size: the same launches per
    step for one instance and for five -- once their list sizes are known,
    the step is twelve launches of the batched build (time step, reset,
    keys, sort, gather, packing, walk, offsets, placement, queue walk, two
    segment sorts) and eight of the evaluations (predictor and corrector:
    pass A, pass B, stage; the packing between them; the density store)."""
    d = wl.taylor_green(nx=40)
    bs = torch.cuda.Stream()
    per_step = []
    for k in (1, 5):
        sims = [_make(d, sph.SPH_MIXED, bs.cuda_stream) for _ in range(k)]
        with sph.Batch(8, bs.cuda_stream) as b:
            b.step(sims)
            l0 = b.launches
            b.step(sims)
            b.step(sims, want_time=True)
            per_step.append((b.launches - l0) / 2)
        for s in sims:
            s.close()
    assert per_step[0] == per_step[1] == 20


def test_batch_argument_errors_change_nothing():
    d = wl.taylor_green(nx=30)
    bs = torch.cuda.Stream()
    s1 = _make(d, sph.SPH_MIXED, bs.cuda_stream)
    s2 = _make(d, sph.SPH_MIXED, bs.cuda_stream)
    before = by_id(s1, FIELDS)
    P = sph.make_params(d["params"], precision=sph.SPH_MIXED, capacity=100)
    empty = sph.Simulation(P, bs.cuda_stream)
    with sph.Batch(2, bs.cuda_stream) as b:
        with pytest.raises(sph.SphError) as e:
            b.step([s1, s1])
        assert e.value.status == sph.SPH_EINVAL
        with pytest.raises(sph.SphError) as e:
            b.step([s1, s2, s1])          # more than max_instances
        assert e.value.status == sph.SPH_EINVAL
        with pytest.raises(sph.SphError) as e:
            b.step([])
        assert e.value.status == sph.SPH_EINVAL
        with pytest.raises(sph.SphError) as e:
            b.step([s1, empty])
        assert e.value.status == sph.SPH_ESTATE
        assert b.launches == 0
    after = by_id(s1, FIELDS)
    for f in FIELDS:
        assert np.array_equal(before[f], after[f]), f
    assert s1.info()["steps"] == 0
    for s in (s1, s2, empty):
        s.close()


def _oracle_after(d, steps):
    P = oracle.params(**d["params"])
    st = oracle.make_state(d["particles"])
    t = oracle.step(P, st, steps)
    return t, st


def test_batched_steps_match_the_oracle():
    """Ten batched PEC steps of three jittered Taylor-Green vortices (two
    mixed, one FP64; the batch's own team sizes) against the oracle's ten
    steps of each, with the single-instance step test's bounds: 1e-4
    (mixed) and 1e-10 (FP64) of each field's magnitude, positions of dx."""
    cases = [(wl.taylor_green(nx=32, jitter=0.1, seed=2, Re=100), sph.SPH_MIXED, 1e-4),
             (wl.taylor_green(nx=32, jitter=0.1, seed=2, Re=100), sph.SPH_FP64, 1e-10),
             (wl.taylor_green(nx=24, jitter=0.1, seed=4, Re=200), sph.SPH_MIXED, 1e-4)]
    bs = torch.cuda.Stream()
    sims = [_make(d, p, bs.cuda_stream) for d, p, _ in cases]
    with sph.Batch(len(sims), bs.cuda_stream) as b:
        t = None
        for _ in range(10):
            t = b.step(sims, want_time=True)
    for q, ((d, prec, tol), sm) in enumerate(zip(cases, sims)):
        tr, st = _oracle_after(d, 10)
        assert abs(t[q] - tr) <= 1e-15 * tr, q
        got = by_id(sm, ["x", "y", "u", "v", "p", "rho"])
        n = st["n"]
        for f in ("x", "y"):
            dxy = got[f] - st[f][:n]
            dxy -= np.round(dxy)                 # unit periodic square
            assert np.abs(dxy).max() <= tol * d["dx"], (q, f)
        for f in ("u", "v", "p", "rho"):
            scale = max(np.abs(st[f][:n]).max(), 1e-30)
            assert np.abs(got[f] - st[f][:n]).max() <= tol * scale, (q, f)
        sm.close()
