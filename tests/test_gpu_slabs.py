"""z-slab decomposition through the C ABI: two processes, each with its own
context for one slab plus ghost planes, exchange the face planes over gloo
(host buffers) once per update; the slabs' fields must equal the
single-domain run bit for bit.  Both processes use cuda:0 (no kernel of one
waits on the other; the exchange is on the host between launches)."""
import os
import socket

import numpy as np
import pytest

from paper_1711_03254_gb300 import workloads as W
from tests.test_gpu_parity import _random_geometry

pytestmark = pytest.mark.gpu

SHAPE = (14, 11, 12)
PARAMS = dict(tau=(0.7, 1.6), G=-1.8, rho_s=0.25, g=(2e-5, -1e-5, 3e-5))


def _case():
    t, r1, r2, u = _random_geometry(SHAPE, 0.15, 123, lo=0.3, hi=0.7)
    return t, r1, r2, u


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, precision, updates, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(0)
    from paper_1711_03254_gb300.slabs import SlabRunner, SlabSim, TorchExchange
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, r1, r2, u = _case()
        s = SlabSim(t, r1, r2, u, PARAMS, rank, world, precision=precision)
        SlabRunner(s, s.L, TorchExchange()).step(updates)
        a, b, v = s.interior_fields()
        np.savez(out, z0=s.z0, z1=s.z1, r1=a, r2=b, u=v)
        s.close()
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_03254_gb300 import build
    build.build()
    from paper_1711_03254_gb300 import lbm as mod
    return mod


@pytest.mark.parametrize("precision,world", [("fp64", 2), ("fp16s", 2), ("fp64", 3)])
def test_slabs_equal_single_domain(lbm, tmp_path, precision, world):
    import torch.multiprocessing as mp
    updates = 50
    ctx = mp.get_context("spawn")
    port = _free_port()
    outs = [str(tmp_path / f"rank{r}.npz") for r in range(world)]
    procs = [ctx.Process(target=_rank, args=(r, world, port, precision, updates, outs[r])) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    t, r1, r2, u = _case()
    nx, ny, nz = SHAPE
    ref = lbm.Sim(nx, ny, nz, [PARAMS], precision=precision, kernel="compact")
    ref.set_geometry(t[None])
    ref.set_fields(r1[None], r2[None], u[None])
    ref.step(updates)
    a, b, v = (x[0] for x in ref.get_fields())
    ref.close()
    for o in outs:
        d = np.load(o)
        z0, z1 = int(d["z0"]), int(d["z1"])
        np.testing.assert_array_equal(d["r1"], a[z0:z1])
        np.testing.assert_array_equal(d["r2"], b[z0:z1])
        np.testing.assert_array_equal(d["u"], v[z0:z1])


def test_split_update_equals_update(lbm):
    """lbm_step_part(0) then (1) on one context is exactly lbm_step(1); parts
    out of order are refused."""
    t, r1, r2, u = _case()
    nx, ny, nz = SHAPE
    sims = []
    for _ in range(2):
        s = lbm.Sim(nx, ny, nz, [PARAMS], precision="fp32", kernel="compact")
        s.set_geometry(t[None])
        s.set_fields(r1[None], r2[None], u[None])
        sims.append(s)
    for _ in range(5):
        sims[0].step(1)
        lbm.lbm_step_part(sims[1].ctx, 0)
        lbm.lbm_step_part(sims[1].ctx, 1)
    np.testing.assert_array_equal(sims[0].get_f(), sims[1].get_f())
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_step_part(sims[1].ctx, 1)
    assert e.value.status == 6
    lbm.lbm_step_part(sims[1].ctx, 0)
    with pytest.raises(lbm.LbmError) as e:
        sims[1].step(1)
    assert e.value.status == 6
    lbm.lbm_step_part(sims[1].ctx, 1)
    for s in sims:
        s.close()


def test_plane_copy_roundtrip_and_sizes(lbm):
    """Plane parts read back what was written; sizes follow the plane's
    non-solid cells; a batch of two instances is refused."""
    t, r1, r2, u = _case()
    nx, ny, nz = SHAPE
    s = lbm.Sim(nx, ny, nz, [PARAMS], precision="fp16s", kernel="compact")
    s.set_geometry(t[None])
    s.set_fields(r1[None], r2[None], u[None])
    s.step(2)
    for z in (0, 5, nz - 1):
        cells = int((t[z] != W.SOLID).sum())
        assert lbm.lbm_plane_bytes(s.ctx, "f_up", z) == cells * 5 * 4
        assert lbm.lbm_plane_bytes(s.ctx, "psi", z) == cells * 8
        for part in ("f_up", "f_down", "psi"):
            a = lbm.lbm_plane_get(s.ctx, part, z)
            lbm.lbm_plane_set(s.ctx, part, z, a[::-1].copy())
            np.testing.assert_array_equal(lbm.lbm_plane_get(s.ctx, part, z), a[::-1])
            lbm.lbm_plane_set(s.ctx, part, z, a)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_plane_bytes(s.ctx, "psi", nz)
    s.close()
    two = lbm.Sim(nx, ny, nz, [PARAMS, PARAMS], precision="fp64", kernel="compact")
    two.set_geometry(np.stack([t, t]))
    two.set_fields(np.stack([r1, r1]), np.stack([r2, r2]), np.stack([u, u]))
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_plane_bytes(two.ctx, "psi", 0)
    assert e.value.status == 1
    two.close()
