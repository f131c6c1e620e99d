"""One domain split into z-slabs, one process (and GPU) per slab.

The update of Eq. 9 reaches one cell in every direction: the streaming of
Eq. 1 moves f* one cell, and the interaction force of Eq. 7 reads psi of the
18 neighbours.  So a slab needs, per update, one ghost plane on either face,
and the exchange is one step per update in two halves:

  1. before the update, the post-collision values that stream across each face:
     the 5 directions with c_z = +1 of the lower neighbour's last plane, and the
     5 with c_z = -1 of the upper neighbour's first plane;
  2. between the density pass and the collision pass, psi of the neighbours'
     face planes (lbm_step_part splits the update there).

Each context holds its slab plus the two ghost planes (periodic in z inside
the context; the ghost cells' own results are meaningless and are
overwritten).  The slab cells then follow the single-domain update bit for
bit, in every storage format.

The transport is a small interface (`Exchange`): `TorchExchange` sends the
planes as byte tensors over torch.distributed (gloo: host memory; NCCL: device
memory, received straight into the receiver's buffer).  The backend that holds
the slab (`SlabSim`, the CUDA library) and the transport are independent, so
the exchange logic runs on CPU with gloo ranks and a stand-in backend.
"""
from __future__ import annotations

from typing import Protocol

import numpy as np

PLANES = ("f_up", "f_down", "psi")


def slab_range(nz: int, rank: int, world: int) -> tuple[int, int]:
    """Planes [z0, z1) of rank's slab: contiguous, sizes differing by at most one."""
    if not (0 <= rank < world) or world > nz:
        raise ValueError("need 0 <= rank < world <= nz")
    return rank * nz // world, (rank + 1) * nz // world


def with_ghosts(a: np.ndarray, z0: int, z1: int) -> np.ndarray:
    """Planes z0 - 1 ... z1 (wrapped) of an array whose first axis is z."""
    nz = a.shape[0]
    idx = [(z0 - 1) % nz] + list(range(z0, z1)) + [z1 % nz]
    return np.ascontiguousarray(a[idx])


class Exchange(Protocol):
    """Point-to-point transport of byte planes between slab neighbours:
    exchange(send_up, send_down, n_lower, n_upper) sends `send_up` to the upper
    neighbour and `send_down` to the lower one, and returns (the lower
    neighbour's send_up, the upper neighbour's send_down) of n_lower and
    n_upper bytes."""

    def exchange(self, send_up: np.ndarray, send_down: np.ndarray, recv_from_lower: int,
                 recv_from_upper: int) -> tuple[np.ndarray, np.ndarray]: ...


class LocalExchange:
    """One slab holding the whole (periodic) domain: it is its own neighbour."""

    def exchange(self, send_up, send_down, recv_from_lower, recv_from_upper):
        return send_up.copy(), send_down.copy()


class TorchExchange:
    """torch.distributed point-to-point (gloo or NCCL process group); ranks
    form a ring along z."""

    def __init__(self, device=None):
        import torch.distributed as dist
        self.dist = dist
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()
        self.device = device  # None: host tensors (gloo); a CUDA device for NCCL

    def exchange(self, send_up, send_down, recv_from_lower, recv_from_upper):
        import torch
        if self.world == 1:
            return send_up.copy(), send_down.copy()
        lower, upper = (self.rank - 1) % self.world, (self.rank + 1) % self.world
        dev = self.device or "cpu"
        su = torch.from_numpy(np.ascontiguousarray(send_up)).to(dev)
        sd = torch.from_numpy(np.ascontiguousarray(send_down)).to(dev)
        ru = torch.empty(recv_from_lower, dtype=torch.uint8, device=dev)
        rd = torch.empty(recv_from_upper, dtype=torch.uint8, device=dev)
        # tag 0: data moving up (+z), tag 1: data moving down; with two ranks the
        # lower and upper neighbour are the same process and the tags keep the
        # two messages apart
        ops = [self.dist.isend(su, upper, tag=0), self.dist.isend(sd, lower, tag=1),
               self.dist.irecv(ru, lower, tag=0), self.dist.irecv(rd, upper, tag=1)]
        for op in ops:
            op.wait()
        return ru.cpu().numpy(), rd.cpu().numpy()


class SlabRunner:
    """Drives the split update of one slab.  `backend` holds the slab with its
    ghost planes (local planes 0 and L + 1) and provides
      plane_get(part, z) -> uint8 array, plane_set(part, z, array),
      plane_bytes(part, z) -> int, step_part(0 | 1)."""

    def __init__(self, backend, interior_planes: int, exchange: Exchange):
        self.b = backend
        self.L = int(interior_planes)
        self.x = exchange

    def _swap(self, up_part: str, down_part: str):
        L, b = self.L, self.b
        # my last plane's upward part goes to the upper neighbour's lower ghost,
        # my first plane's downward part to the lower neighbour's upper ghost
        got_up, got_down = self.x.exchange(b.plane_get(up_part, L), b.plane_get(down_part, 1),
                                           b.plane_bytes(up_part, 0), b.plane_bytes(down_part, L + 1))
        b.plane_set(up_part, 0, got_up)
        b.plane_set(down_part, L + 1, got_down)

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self._swap("f_up", "f_down")
            self.b.step_part(0)
            self._swap("psi", "psi")
            self.b.step_part(1)


class SlabSim:
    """The CUDA library as a slab backend: a context of nx x ny x (L + 2)
    cells for rank's slab of a global [nz, ny, nx] problem (one instance)."""

    def __init__(self, t, r1, r2, u, params, rank: int, world: int, precision="fp64", eq_order=0, wall_model=2):
        from paper_1711_03254_gb300 import lbm
        self.lbm = lbm
        nz, ny, nx = t.shape
        self.z0, self.z1 = slab_range(nz, rank, world)
        self.L = self.z1 - self.z0
        g = lambda a: with_ghosts(a, self.z0, self.z1)
        self.sim = lbm.Sim(nx, ny, self.L + 2, [params], precision=precision, eq_order=eq_order,
                           wall_model=wall_model, kernel="compact")
        self.sim.set_geometry(g(t)[None])
        self.sim.set_fields(g(r1)[None], g(r2)[None], g(u)[None])

    def plane_bytes(self, part, z):
        return self.lbm.lbm_plane_bytes(self.sim.ctx, part, z)

    def plane_get(self, part, z):
        return self.lbm.lbm_plane_get(self.sim.ctx, part, z)

    def plane_set(self, part, z, a):
        self.lbm.lbm_plane_set(self.sim.ctx, part, z, a)

    def step_part(self, p):
        self.lbm.lbm_step_part(self.sim.ctx, p)

    def interior_fields(self):
        """(rho1, rho2, u) of the slab's own planes, [L, ny, nx] (u [..., 3])."""
        r1, r2, u = self.sim.get_fields()
        return r1[0, 1:-1], r2[0, 1:-1], u[0, 1:-1]

    def close(self):
        self.sim.close()
