"""Shared test helpers: GPU availability, id alignment and the
condition-aware parity norm."""
import numpy as np
import pytest

FP64_TOL = 1e-12   # max_i |gpu - oracle| / max_i S_i, FP64 path
MIXED_TOL = 2e-5   # same norm, FP32 pair arithmetic


def cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def stream_handle():
    import torch
    return torch.cuda.current_stream().cuda_stream


def by_id(sim, fields):
    """Read fields from a Simulation, reordered by particle id."""
    ids = sim.read("id")
    order = np.argsort(ids, kind="stable")
    out = {"id": ids[order]}
    for f in fields:
        out[f] = sim.read(f)[order]
    return out


def norm(a, b, scale):
    """max_i |a_i - b_i| / max_i S_i (S_i = sum of |terms| of b_i)."""
    s = float(np.max(scale)) if len(scale) else 1.0
    if s == 0.0:
        s = 1.0
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / s


def neighbour_sets_by_id(sim):
    ids = sim.read("id")
    off = sim.read("neigh_off")
    nid = sim.read("neigh_id")
    sets = {}
    for k, i in enumerate(ids):
        sets[int(i)] = np.sort(nid[off[k]:off[k + 1]])
    return sets
