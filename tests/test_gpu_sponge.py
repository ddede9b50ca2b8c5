"""The upstream sponge of the periodic cylinder stand-in (sph_params
sponge_width): after one PEC step the positions are those of the run
without it and u, v, p are relaxed towards (U_ref, 0, 0) by the stated
fraction min(1, 10 U_ref dt / w s^2), s the depth into the layer."""
import numpy as np
import pytest

from paper_2107_01276_gb300 import sph
from paper_2107_01276_gb300 import workloads as wl
from tests.helpers import by_id, cuda_ok, stream_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not cuda_ok():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("precision", [sph.SPH_FP64, sph.SPH_MIXED])
def test_sponge_relaxes_by_the_stated_fraction(precision):
    d = wl.taylor_green(nx=40, jitter=0.1, seed=8)
    n = len(d["particles"]["x"])
    w = 0.3
    out = {}
    for width in (0.0, w):
        P = sph.make_params(d["params"], precision=precision, capacity=n,
                            sponge_width=width)
        s = sph.Simulation(P, stream_handle())
        s.load(d["particles"])
        s.step(1)
        out[width] = by_id(s, ["x", "y", "u", "v", "p"])
        out[width]["dt"] = s.info()["dt"]
        s.close()
    a, b = out[0.0], out[w]
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["y"], b["y"])
    U = d["params"].get("U_ref", 1.0)
    s_ = np.clip((d["params"]["lo"][0] + w - a["x"]) / w, 0.0, None)
    k = np.minimum(1.0, 10.0 * U * a["dt"] / w * s_ * s_)
    inside = s_ > 0
    assert inside.sum() > 100 and (~inside).sum() > 100
    np.testing.assert_allclose(b["u"], a["u"] + (U - a["u"]) * k, rtol=0, atol=1e-14)
    np.testing.assert_allclose(b["v"], a["v"] - a["v"] * k, rtol=0, atol=1e-14)
    np.testing.assert_allclose(b["p"], a["p"] - a["p"] * k, rtol=0,
                               atol=1e-14 * np.abs(a["p"]).max())
    # outside the layer nothing changes
    for f in ("u", "v", "p"):
        assert np.array_equal(a[f][~inside], b[f][~inside])
