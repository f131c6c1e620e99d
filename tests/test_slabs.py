"""Host logic of the z-slab decomposition on CPU (gloo ranks, no GPU): the
slab split, the ghost planes of the local geometry, and the exchange of the
face planes between neighbours in the order of one update (crossing
distributions, density pass, psi, collision pass)."""
import os
import socket

import numpy as np
import pytest

from paper_1711_03254_gb300.slabs import LocalExchange, SlabRunner, slab_range, with_ghosts


@pytest.mark.parametrize("nz,world", [(8, 1), (8, 2), (9, 2), (10, 3), (7, 7)])
def test_slab_range_tiles_planes(nz, world):
    r = [slab_range(nz, k, world) for k in range(world)]
    assert r[0][0] == 0 and r[-1][1] == nz
    assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
    sizes = [b - a for a, b in r]
    assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slab_range(3, 0, 4)


def test_with_ghosts_wraps():
    a = np.arange(6)[:, None] * np.ones((6, 2))
    g = with_ghosts(a, 0, 3)
    assert list(g[:, 0]) == [5, 0, 1, 2, 3]
    g = with_ghosts(a, 4, 6)
    assert list(g[:, 0]) == [3, 4, 5, 0]
    g = with_ghosts(a, 0, 6)
    assert list(g[:, 0]) == [5, 0, 1, 2, 3, 4, 5, 0]


class PlaneStore:
    """Stand-in backend: the planes of a slab with ghosts as byte arrays whose
    content names (part, global plane, generation); the generation is the
    number of completed updates, and planes of different z have different
    lengths (as the non-solid cell counts of a real geometry do)."""

    def __init__(self, nz, z0, z1):
        self.nz, self.z0, self.z1 = nz, z0, z1
        self.L = z1 - z0
        self.gen = 0
        self.log = []
        self.planes = {}
        for part in ("f_up", "f_down", "psi"):
            for zl in range(self.L + 2):
                self.planes[(part, zl)] = self._content(part, self._global(zl), -1)

    def _global(self, zl):
        return (self.z0 - 1 + zl) % self.nz

    @staticmethod
    def _size(part, zg):
        return 3 + zg % 4 + (2 if part == "psi" else 0)

    def _content(self, part, zg, gen):
        head = np.array([("f_up", "f_down", "psi").index(part), zg, gen % 256], dtype=np.uint8)
        return np.concatenate([head, np.full(self._size(part, zg) - 3, 7, np.uint8)])

    def plane_bytes(self, part, zl):
        return self._size(part, self._global(zl))

    def plane_get(self, part, zl):
        assert 1 <= zl <= self.L, "only slab planes are sent"
        # f of the last update, psi of the density pass in progress
        return self._content(part, self._global(zl), self.gen).copy()

    def plane_set(self, part, zl, a):
        assert zl in (0, self.L + 1), "only ghost planes are received"
        self.planes[(part, zl)] = np.asarray(a).copy()
        self.log.append(("set", part, zl))

    def step_part(self, p):
        self.log.append(("part", p))
        if p == 1:
            self.gen += 1


def _check_ghosts(store, updates):
    lower = store.planes[("f_up", 0)]
    upper = store.planes[("f_down", store.L + 1)]
    zl, zu = (store.z0 - 1) % store.nz, store.z1 % store.nz
    # the ghost planes hold the neighbours' face planes of the last exchange
    assert list(lower[:3]) == [0, zl, (updates - 1) % 256] and len(lower) == store._size("f_up", zl)
    assert list(upper[:3]) == [1, zu, (updates - 1) % 256] and len(upper) == store._size("f_down", zu)
    for zg, zloc in ((zl, 0), (zu, store.L + 1)):
        p = store.planes[("psi", zloc)]
        assert list(p[:3]) == [2, zg, (updates - 1) % 256]
    # order within each update: f ghosts, density pass, psi ghosts, collision pass
    per = [("set", "f_up", 0), ("set", "f_down", store.L + 1), ("part", 0),
           ("set", "psi", 0), ("set", "psi", store.L + 1), ("part", 1)]
    assert store.log == per * updates


def test_single_slab_is_its_own_neighbour():
    s = PlaneStore(6, 0, 6)
    SlabRunner(s, s.L, LocalExchange()).step(3)
    _check_ghosts(s, 3)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, nz, updates, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from paper_1711_03254_gb300.slabs import TorchExchange
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        z0, z1 = slab_range(nz, rank, world)
        s = PlaneStore(nz, z0, z1)
        SlabRunner(s, s.L, TorchExchange()).step(updates)
        _check_ghosts(s, updates)
        q.put((rank, "ok"))
    except Exception as e:  # reported to the parent
        q.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,nz", [(2, 7), (3, 9), (2, 2)])
def test_exchange_over_gloo_ranks(world, nz):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, nz, 4, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res == {r: "ok" for r in range(world)}, res
