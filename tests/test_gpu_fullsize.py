"""Parity at the benchmark's full size (graded 1:250 strip, ~1.08M
particles) in the configuration bench.py times: cell keys for every
particle, neighbour sets and right-hand-side values for a random sample of
particles that the oracle evaluates one by one."""
import numpy as np
import pytest

import oracle
from paper_2107_01276_gb300 import sph
from paper_2107_01276_gb300 import workloads as wl
from tests.helpers import FP64_TOL, MIXED_TOL, cuda_ok, norm, stream_handle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

RHS_FIELDS = ("rho", "beta", "pavg", "drx", "dry", "dpdt", "dudt", "dvdt")


@pytest.fixture(scope="module")
def graded():
    if not cuda_ok():
        pytest.skip("no CUDA device")
    return wl.graded_strip(n_target=1 << 20, ratio=250.0)


def _sparse_csr(n, rows, off_r, nbr_r):
    """Full-size CSR holding lists only for the particles in ``rows``."""
    cnt = np.zeros(n, np.int64)
    cnt[rows] = np.diff(off_r)
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum(cnt)
    nbr = np.zeros(off[-1], np.int32)
    for k, r in enumerate(rows):
        nbr[off[r]:off[r + 1]] = nbr_r[off_r[k]:off_r[k + 1]]
    return off.astype(np.int32), nbr


def _oracle_sampled(d, sample, dt):
    """Pass A on the sample and its neighbours, pass B on the sample."""
    pt = d["particles"]
    P = oracle.params(**d["params"])
    n = len(pt["x"])
    xs = lambda idx: (pt["x"][idx], pt["y"][idx], pt["h"][idx])
    o1, n1 = oracle.neighbors_cross(P, *xs(sample), pt["x"], pt["y"], pt["h"])
    U = np.unique(np.concatenate([sample, n1]))
    oU, nU = oracle.neighbors_cross(P, *xs(U), pt["x"], pt["y"], pt["h"])
    off, nbr = _sparse_csr(n, U, oU, nU)
    with np.errstate(all="ignore"):
        a = oracle.pass_a(P, pt["x"], pt["y"], pt["h"], pt["m"], pt["p"],
                          off, nbr)
        offs, nbrs = _sparse_csr(n, sample, o1, n1)
        b = oracle.pass_b(P, dt, pt["x"], pt["y"], pt["h"], pt["m"], pt["p"],
                          pt["u"], pt["v"], offs, nbrs, a)
    out = {k: v[sample] for k, v in b.items()}
    for k in ("rho", "beta", "pavg", "drx", "dry", "nnb", "s_rho", "s_beta",
              "s_pavg", "s_drx", "s_dry"):
        out[k] = a[k][sample]
    return (o1, n1), out


@pytest.mark.parametrize("precision,tol", [(sph.SPH_MIXED, MIXED_TOL),
                                           (sph.SPH_FP64, FP64_TOL)])
def test_full_size_sampled_parity(graded, precision, tol):
    d = graded
    pt = d["particles"]
    n = len(pt["x"])
    P = sph.make_params(d["params"], precision=precision,
                        capacity=int(n * 1.1) + 16)
    sim = sph.Simulation(P, stream_handle())
    sim.load(pt)
    sim.rhs()
    ids = sim.read("id")
    pos = np.empty(n, np.int64)
    pos[ids] = np.arange(n)
    # keys of every particle, bit-exact
    key = sim.read("cellkey")
    okey, _ = oracle.cell_keys(oracle.params(**d["params"]),
                               sim.info()["c0"], pt["x"], pt["y"], pt["h"])
    assert np.array_equal(key[pos], okey)
    # sample, weighted towards the graded transitions by taking it uniform
    # in index (columns run from coarse to fine)
    rng = np.random.default_rng(17)
    sample = np.sort(rng.choice(n, 160, replace=False))
    dt = oracle.dt(oracle.params(**d["params"]), pt["h"])
    (o1, n1), ref = _oracle_sampled(d, sample, dt)
    off = sim.read("neigh_off")
    nid = sim.read("neigh_id")
    for k, i in enumerate(sample):
        p = pos[i]
        got = np.sort(nid[off[p]:off[p + 1]])
        assert np.array_equal(got, n1[o1[k]:o1[k + 1]]), i
    got = {f: sim.read(f)[pos[sample]] for f in RHS_FIELDS}
    nnb = sim.read("nnb")[pos[sample]]
    assert np.array_equal(nnb, ref["nnb"])
    for f in RHS_FIELDS:
        e = norm(got[f], ref[f], ref["s_" + f])
        assert e <= tol, (f, e)
    sim.close()
