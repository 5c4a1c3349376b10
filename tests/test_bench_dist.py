"""Host logic of bench.py's multi-GPU mode, run as two gloo ranks on the CPU.

N ranks cluster independent seeded point sets (weak scaling, no data-path
collective); the whole-job time per clustering is the slowest rank's timed
total divided by the clusterings all ranks ran; the reference arm runs on rank
0 only.
"""
import importlib.util
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    r, w, local = b.dist_env()
    t_local = [12.0, 20.0][rank]              # ms over `steps` timed clusterings
    value, per_step = b.job_ms_per_clustering(t_local, 4, w, dist, "cpu")
    e2e = b.reduce_max([3.0, 5.0][rank], dist, "cpu") / w
    dist.barrier()
    q.put((r, w, local, value, per_step, e2e, b.reference_runs_on(r)))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, w, local, value, per_step, e2e, ref) in enumerate(out):
        assert (rank, w, local) == (r, 2, r)
        assert value == pytest.approx(20.0 / (4 * 2))     # slowest rank, all clusterings
        assert per_step == pytest.approx(20.0 / 4)
        assert e2e == pytest.approx(5.0 / 2)
        assert ref == (rank == 0)


def test_single_rank_identity():
    b = _bench()
    assert b.job_ms_per_clustering(8.0, 4, 1, None, "cpu") == (2.0, 2.0)
    assert b.reduce_max(1.5, None, "cpu") == 1.5


def test_ranks_get_independent_inputs():
    b = _bench()
    a0, a1, again = b.make_input(0), b.make_input(1), b.make_input(0)
    assert a0.X.shape == a1.X.shape == (200_000, 3)
    assert not np.array_equal(a0.X, a1.X)
    assert np.array_equal(a0.X, again.X)
