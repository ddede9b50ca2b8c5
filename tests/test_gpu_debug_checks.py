"""The debug build (the library compiled with SPH_DEBUG): device-side
bounds checks on neighbour-list gathers, the list build's cell ranges, the
sort's gather and the compaction writes count a failure and skip the
access instead of trapping.  A run of small cases -- the per-particle team
walk, cell tiles with rows that overflow the first build's staging, and a
cylinder with walls, splits and merges -- counts no failure in the debug
library and gives the release library's states bit for bit.  The debug
library runs in a child process (SPH_GB300_DEBUG_LIB=1)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from tests.helpers import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FIELDS = ("x", "y", "u", "v", "p", "m", "h", "id")


def run_cases():
    """The cases' final states (the same calls in either library)."""
    import torch

    from paper_2107_01276_gb300 import sph
    from paper_2107_01276_gb300 import workloads as wl
    st = torch.cuda.current_stream().cuda_stream
    out = {}

    def sim(d, cap):
        P = sph.make_params(d["params"], precision=sph.SPH_MIXED, capacity=cap)
        s = sph.Simulation(P, st)
        s.load(d["particles"])
        return s

    d = wl.taylor_green(nx=40, jitter=0.1, seed=31)
    s = sim(d, 1600)
    s.step(3)
    out["tgv"] = {f: s.read(f) for f in FIELDS}
    s.close()
    d = wl.perturbed(nx=280, ny=260, h_ratio=2.0, hdx=1.7, seed=11)
    s = sim(d, len(d["particles"]["x"]))
    s.step(2)
    out["tiles"] = {f: s.read(f) for f in FIELDS}
    s.close()
    d = wl.cylinder(Re=40.0, background="rings")
    s = sim(d, 400000)
    s.load(d["walls"], kind=sph.SPH_WALL)
    s.load(d["background_rings"], kind=sph.SPH_BACKGROUND)
    merged = 0
    for _ in range(3):
        merged += s.adapt()["n_merged"]
        s.step(1)
    out["cylinder"] = {f: s.read(f) for f in FIELDS}
    out["cylinder"]["merged"] = np.array([merged])
    s.close()
    return out


def main(path):
    """Child process: run the cases in the loaded library and save them with
    the library's kind and failure count."""
    from paper_2107_01276_gb300 import sph
    sph.lib()
    sph.debug_failures()   # start from zero
    out = run_cases()
    flat = {"%s.%s" % (c, f): v for c, d in out.items() for f, v in d.items()}
    flat["debug_build"] = np.array([int(sph.debug_build())])
    flat["failures"] = np.array([sph.debug_failures()])
    np.savez(path, **flat)


def test_debug_build_counts_no_failure_and_matches_release(tmp_path):
    if not cuda_ok():
        pytest.skip("no CUDA device")
    path = str(tmp_path / "debug.npz")
    env = dict(os.environ, SPH_GB300_DEBUG_LIB="1")
    code = ("import sys; sys.path.insert(0, %r); "
            "import tests.test_gpu_debug_checks as t; t.main(%r)" % (ROOT, path))
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stderr[-3000:]
    dbg = np.load(path)
    assert int(dbg["debug_build"][0]) == 1
    assert int(dbg["failures"][0]) == 0
    from paper_2107_01276_gb300 import sph
    assert not sph.debug_build() and sph.debug_failures() == 0
    rel = run_cases()
    assert int(rel["cylinder"]["merged"][0]) > 0
    for c, d in rel.items():
        for f, v in d.items():
            assert np.array_equal(v, dbg["%s.%s" % (c, f)]), (c, f)
