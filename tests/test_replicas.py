"""Multi-rank host logic on CPU (gloo, world size 2 and 3): the instance split,
the gather of per-instance results and the max over ranks used for timing."""
import os
import socket

import numpy as np
import pytest

from paper_1711_03254_gb300.replicas import shard


@pytest.mark.parametrize("n,world", [(0, 2), (1, 2), (7, 2), (7, 3), (16, 8), (5, 8)])
def test_shard_tiles_units(n, world):
    blocks = [shard(n, r, world) for r in range(world)]
    assert [i for b in blocks for i in b] == list(range(n))
    sizes = [len(b) for b in blocks]
    assert max(sizes) - min(sizes) <= 1
    assert sizes == sorted(sizes, reverse=True)


def test_shard_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard(4, 2, 2)
    with pytest.raises(ValueError):
        shard(4, 0, 0)


def _unit_result(k):
    # a per-instance result computed on the host: the sharp-interface 1|2|1
    # channel velocity maximum for instance k's viscosity ratio
    from tests import analytic  # noqa: F401  (import check on every rank)
    nu1, nu2 = 0.1, 0.1 / (1.0 + k)
    h, a, g = 30.0, 15.0, 1e-6
    umax = g * (h * h - a * a) / (2 * nu1) + g * a * a / (2 * nu2)
    return [float(k), umax, nu2]


def _worker(rank, world, port, n, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from paper_1711_03254_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = replicas.shard(n, rank, world)
        rows = np.array([_unit_result(k) for k in mine]).reshape(len(mine), 3)
        allrows = replicas.gather_units(rows, n)
        slowest = replicas.max_over_ranks(0.5 + rank)
        q.put((rank, allrows, slowest))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("world,n", [(2, 7), (3, 4)])
def test_gather_and_max_over_gloo_ranks(world, n):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = np.array([_unit_result(k) for k in range(n)])
    for rank, rows, slowest in got:
        np.testing.assert_array_equal(rows, want)
        assert slowest == 0.5 + world - 1
