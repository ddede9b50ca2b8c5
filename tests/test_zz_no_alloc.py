"""The no-allocation entry point sph_cell_sort_noalloc, for callers that
cannot allocate device memory themselves (for example a solver inside a
host application that owns all device memory through its own pool).  Its
keys and order must equal those of the context's own rebuild and the
oracle's keys, on the single-block sort (small sets) and on the multi-tile
sort whose counts and scan sums live in the fixed scratch array (up to its
262144-particle limit).  This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
from paper_2107_01276_gb300 import sph
from paper_2107_01276_gb300 import workloads as wl
from tests.helpers import cuda_ok, stream_handle


def _reference(d):
    """Keys and order from the existing path: a context, sph_rhs, then
    SPH_F_CELLKEY / SPH_F_ID (ids are the input indices)."""
    n = len(d["particles"]["x"])
    P = sph.make_params(d["params"], precision=sph.SPH_FP64, capacity=n)
    sim = sph.Simulation(P, stream_handle())
    sim.load(d["particles"])
    sim.rhs()
    out = sim.read("cellkey"), sim.read("id"), sim.info()["c0"]
    sim.close()
    return out


def _noalloc(d, c0):
    import torch
    pt = d["particles"]
    n = len(pt["x"])
    P = sph.make_params(d["params"], precision=sph.SPH_FP64, capacity=n,
                        cell_c0=c0)
    dev = {k: torch.tensor(pt[k], dtype=torch.float64, device="cuda")
           for k in ("x", "y", "h")}
    key = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    st = sph.cell_sort_noalloc(P, n, dev["x"].data_ptr(), dev["y"].data_ptr(),
                               dev["h"].data_ptr(), key.data_ptr(),
                               perm.data_ptr(), stream_handle())
    assert st == sph.SPH_OK, sph.last_error()
    torch.cuda.synchronize()
    return key.cpu().numpy().view(np.uint64), perm.cpu().numpy().astype(np.int64)


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["small", "multi_tile"])
def test_no_alloc_matches_context_rebuild_and_oracle_twice(case):
    """Each set twice in a row (the array keeps the previous call's
    contents): keys and order equal the context's, keys equal the
    oracle's cell keys of the same particles."""
    if not cuda_ok():
        pytest.skip("no CUDA device")
    if case == "small":      # single-block sorts (at most 16384 particles)
        sets = [wl.perturbed(nx=61, ny=47, h_ratio=4.0, seed=21),
                wl.graded_strip(n_target=6000, ratio=16.0)]
    else:                    # tiled radix sorts: ~100k and the 262144 limit
        sets = [wl.graded_strip(n_target=100000, ratio=64.0),
                wl.perturbed(nx=512, ny=512, h_ratio=3.0, seed=22)]
    for d in sets:
        pt = d["particles"]
        key_ref, id_ref, c0 = _reference(d)
        okey, _ = oracle.cell_keys(oracle.params(**d["params"]), c0, pt["x"],
                                   pt["y"], pt["h"])
        for _ in range(2):
            got_key, got_perm = _noalloc(d, c0)
            assert np.array_equal(got_key, key_ref)
            assert np.array_equal(got_perm, id_ref)
            assert np.array_equal(got_key, okey[got_perm])


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    """Checked before any device work, so no GPU is needed; the reason is
    reported through sph_last_error(NULL)."""
    d = wl.taylor_green(nx=10)
    P = sph.make_params(d["params"], cell_c0=0.3)
    st = sph.cell_sort_noalloc(P, (1 << 18) + 1, 0, 0, 0, 0, 0)
    assert st == sph.SPH_EINVAL
    assert "262144" in sph.last_error()
    st = sph.cell_sort_noalloc(P, 10, 0, 0, 0, 0, 0)   # NULL arrays
    assert st == sph.SPH_EINVAL
    assert "NULL" in sph.last_error()
