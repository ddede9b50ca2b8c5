"""The multi-GPU form is replicas only (one independent simulation per
rank, no data-path collective): bench.py's whole-job figure is the units
all ranks processed over the slowest rank's time.  Checked here with two
gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 1.5 + r seconds for 100 (1 + 2 r) particle-steps
        t, u = bench.replica_totals(dist, 1.5 + rank, 100.0 * (1 + 2 * rank),
                                    device="cpu")
        out.put((rank, t, u))
    finally:
        dist.destroy_process_group()


def test_replica_totals_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    # slowest rank's time, all ranks' units, on every rank
    assert got == [(0, 2.5, 400.0), (1, 2.5, 400.0)]


def test_replica_totals_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_totals(None, 3.0, 7) == (3.0, 7.0)
