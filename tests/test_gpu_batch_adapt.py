"""sph_batch_adapt: the adaptations of several contexts in lockstep (one
host synchronisation of all of them per phase) leave every context where
sph_adapt on it alone leaves it, bit for bit: a cylinder with walls and a
ring background, a refinement strip in both precisions, an adaptive
Taylor-Green vortex whose background is rebuilt inside every second call,
and a context whose split children exceed its capacity, which fails as it
does alone while the others go on."""
import numpy as np
import pytest

from paper_2107_01276_gb300 import sph
from paper_2107_01276_gb300 import workloads as wl
from tests.helpers import cuda_ok

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "u", "v", "p", "rho", "m", "h", "mmin", "mmax", "id")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not cuda_ok():
        pytest.skip("no CUDA device")


def _strip(seed):
    d = wl.perturbed(nx=30, ny=30, h_ratio=1.0, jitter=0.1, hdx=1.2,
                     periodic=(1, 1), seed=seed)
    dx = d["dx"]
    g = (np.arange(60) + 0.5) / 60
    X, Y = np.meshgrid(g, g, indexing="xy")
    bg = {"x": X.ravel(), "y": Y.ravel(), "h": np.full(X.size, 1.2 / 60)}
    bg["ds"] = np.where(bg["x"] < 0.5, 0.5 * dx, dx)
    return d, bg


def _cases():
    """(name, make(stream) -> Simulation) of the mix."""
    def cyl(stream):
        d = wl.cylinder(Re=40.0, background="rings")
        P = sph.make_params(d["params"], precision=sph.SPH_MIXED, capacity=400000)
        s = sph.Simulation(P, stream)
        s.load(d["particles"])
        s.load(d["walls"], kind=sph.SPH_WALL)
        s.load(d["background_rings"], kind=sph.SPH_BACKGROUND)
        return s

    def strip(precision, seed, cap=20000):
        def make(stream):
            d, bg = _strip(seed)
            P = sph.make_params(d["params"], precision=precision, capacity=cap)
            s = sph.Simulation(P, stream)
            s.load(d["particles"])
            s.load(bg, kind=sph.SPH_BACKGROUND)
            return s
        return make

    def tga(stream):
        d = wl.taylor_green_adaptive(nx=30, Re=100.0)
        pr = dict(d["params"], n_bg=2)
        n = len(d["particles"]["x"])
        P = sph.make_params(pr, precision=sph.SPH_MIXED, capacity=8 * n,
                            bg_capacity=200000)
        s = sph.Simulation(P, stream)
        s.load(d["particles"])
        s.load(d["region"], kind=sph.SPH_REGION)
        s.load(d["background"], kind=sph.SPH_BACKGROUND)
        s.background()
        return s

    return [("cylinder", cyl), ("strip64", strip(sph.SPH_FP64, 21)),
            ("strip32", strip(sph.SPH_MIXED, 22)), ("tg-adaptive", tga)]


def _state(sim):
    return {f: sim.read(f) for f in FIELDS}


def _equal(a, b):
    return all(np.array_equal(a[f], b[f]) for f in FIELDS)


@pytest.mark.parametrize("shared_stream", [False, True])
def test_batch_adapt_equals_alone(shared_stream):
    import torch
    cases = _cases()
    own = [torch.cuda.Stream() for _ in cases]
    one = torch.cuda.Stream()
    solo = [make(st.cuda_stream) for (_, make), st in zip(cases, own)]
    mix = [make(one.cuda_stream if shared_stream else st.cuda_stream)
           for (_, make), st in zip(cases, own)]
    b = sph.Batch(len(mix), torch.cuda.current_stream().cuda_stream)
    split = merged = 0
    for rnd in range(3):
        zs = [s.adapt() for s in solo]
        zb = b.adapt(mix)
        for (name, _), a, c in zip(cases, zs, zb):
            assert a == c, (name, rnd)
        split += sum(z["n_split"] for z in zs)
        merged += sum(z["n_merged"] for z in zs)
        for s in solo + mix:
            s.step(1)
    assert split > 0 and merged > 0
    for (name, _), s, m in zip(cases, solo, mix):
        assert _equal(_state(s), _state(m)), name
        assert s.info()["n"] == m.info()["n"]
    b.close()
    for s in solo + mix:
        s.close()


def test_batch_adapt_with_batch_steps_equals_alone():
    """Adaptation and steps both batched (sph_batch_adapt, then
    sph_batch_step with each context's team sizes fixed) against
    sph_adapt and sph_step alone."""
    import torch
    cases = _cases()[1:3]
    own = [torch.cuda.Stream() for _ in cases]
    solo = [make(st.cuda_stream) for (_, make), st in zip(cases, own)]
    mix = [make(st.cuda_stream) for (_, make), st in zip(cases, own)]
    for s in solo + mix:
        s.set_tuning(team_a=1, team_b=1)
    b = sph.Batch(len(mix), torch.cuda.current_stream().cuda_stream)
    for _ in range(3):
        for s in solo:
            s.adapt()
            s.step(1)
        b.adapt(mix)
        b.step(mix)
    for (name, _), s, m in zip(cases, solo, mix):
        assert _equal(_state(s), _state(m)), name
    b.close()
    for s in solo + mix:
        s.close()


def test_failed_context_stops_alone_and_the_others_go_on():
    import torch
    d, bg = _strip(23)
    n = len(d["particles"]["x"])

    def make(cap, stream):
        P = sph.make_params(d["params"], precision=sph.SPH_FP64, capacity=cap)
        s = sph.Simulation(P, stream)
        s.load(d["particles"])
        s.load(bg, kind=sph.SPH_BACKGROUND)
        return s

    st = [torch.cuda.Stream() for _ in range(4)]
    tight_alone = make(n + 10, st[0].cuda_stream)
    with pytest.raises(sph.SphError) as e:
        tight_alone.adapt()
    assert e.value.status == sph.SPH_ECAPACITY
    ok_alone = make(20000, st[1].cuda_stream)
    z_ok = ok_alone.adapt()
    tight = make(n + 10, st[2].cuda_stream)
    ok = make(20000, st[3].cuda_stream)
    b = sph.Batch(2, torch.cuda.current_stream().cuda_stream)
    out = b.adapt([tight, ok], errors="return")
    assert out[0][0] == sph.SPH_ECAPACITY and "capacity" in out[0][1]
    assert out[1] == z_ok
    assert _equal(_state(ok), _state(ok_alone))
    assert _equal(_state(tight), _state(tight_alone))
    with pytest.raises(sph.SphError) as e:
        b.adapt([ok, tight])
    assert e.value.status == sph.SPH_ECAPACITY
    # argument errors: nothing runs
    n_before = ok.info()["n"]
    with pytest.raises(sph.SphError) as e:
        b.adapt([ok, ok])
    assert e.value.status == sph.SPH_EINVAL
    with pytest.raises(sph.SphError) as e:
        b.adapt([ok, tight, ok_alone])    # more than max_instances
    assert e.value.status == sph.SPH_EINVAL
    assert ok.info()["n"] == n_before
    b.close()
    for s in (tight_alone, ok_alone, tight, ok):
        s.close()
