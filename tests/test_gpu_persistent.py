"""The persistent compact update (LBM_KERNEL_PERSISTENT): n updates of the
compact two-pass update in one cooperative launch with grid-wide barriers.

It runs the same per-cell code as the two-launch compact update (loads of data
written in the same launch go through L2), so the states must agree bit for
bit: fields and distributions, after any number of updates, over ragged grids,
batches, both equilibria, the third-order regularisation, every wall model and
INLET/OUTLET planes; in the steady-state loop too.  The failure path: with a
barrier that waits for an arrival that never comes, every block gives up
after the bound and the host reports LBM_ERR_TIMEOUT, and the context stays
usable.  A timing comparison on batched small instances is printed."""
import time

import numpy as np
import pytest

from paper_1711_03254_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_03254_gb300 import build
    build.build()
    from paper_1711_03254_gb300 import lbm as mod
    return mod


def _geometry(shape, frac, seed, inlet_outlet=False):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    t = np.where(rng.random((nz, ny, nx)) < frac, W.SOLID, W.FLUID).astype(np.uint8)
    if inlet_outlet:
        t[:, :, 0] = np.where(t[:, :, 0] == W.SOLID, W.SOLID, W.INLET)
        t[:, :, nx - 1] = np.where(t[:, :, nx - 1] == W.SOLID, W.SOLID, W.OUTLET)
    r1 = np.where(t == W.SOLID, 0.0, rng.uniform(0.3, 0.7, t.shape))
    r2 = np.where(t == W.SOLID, 0.0, rng.uniform(0.3, 0.7, t.shape))
    u = rng.uniform(-0.03, 0.03, t.shape + (3,))
    u[t == W.SOLID] = 0
    return t, r1, r2, u


def _run(lbm, kernel, shape, params, geo, steps, precision, **cfg):
    nx, ny, nz = shape
    B = len(params)
    sim = lbm.Sim(nx, ny, nz, params, precision=precision, kernel=kernel, **cfg)
    sim.set_geometry(np.stack([g[0] for g in geo]))
    sim.set_fields(np.stack([g[1] for g in geo]), np.stack([g[2] for g in geo]), np.stack([g[3] for g in geo]))
    for n in steps:
        sim.step(n)
    out = sim.get_fields(), sim.get_f()
    sim.close()
    return out


def _same(a, b):
    (fa, da), (fb, db) = a, b
    return all(np.array_equal(x, y, equal_nan=True) for x, y in zip(fa, fb)) and np.array_equal(da, db, equal_nan=True)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s", "bf16s"])
@pytest.mark.parametrize("shape", [(6, 5, 7), (33, 3, 2), (40, 19, 13)])
@pytest.mark.parametrize("cfg", [dict(), dict(eq_order=1, wall_model=0), dict(reg_order=3, wall_model=3),
                                 dict(eq_order=1, wall_model=1)])
def test_bitwise_equal_to_compact(lbm, precision, shape, cfg):
    geo = [_geometry(shape, 0.2, 3 + sum(shape) + k) for k in range(3)]
    params = [dict(tau=(0.6 + 0.1 * k, 1.4), G=-1.5, rho_s=0.2 - 0.1 * k, g=(1e-4, 0, 2e-5)) for k in range(3)]
    for steps in ([7], [1, 2, 3]):
        a = _run(lbm, "compact", shape, params, geo, steps, precision, **cfg)
        b = _run(lbm, "persistent", shape, params, geo, steps, precision, **cfg)
        assert _same(a, b), (steps, cfg)


@pytest.mark.parametrize("precision", ["fp64", "fp16s"])
def test_inlet_outlet_and_large_instance(lbm, precision):
    """Beyond one wave of resident threads (76 800 cells) the blocks stride over
    the items and look the neighbours up every update."""
    shape = (64, 40, 30)
    geo = [_geometry(shape, 0.15, 21, inlet_outlet=True)]
    p = [dict(tau=(0.7, 1.6), G=-1.2, rho_s=-0.2, rho_in=(0.2, 0.8), u_in=(0.02, 0, 0))]
    a = _run(lbm, "compact", shape, p, geo, [20], precision)
    b = _run(lbm, "persistent", shape, p, geo, [20], precision)
    assert _same(a, b)


def test_steady_loop_equal_to_compact(lbm):
    t, r1, r2, u = W.droplet(24, 24, 24, 6.0)
    out = []
    for kernel in ("compact", "persistent"):
        sim = lbm.Sim(24, 24, 24, [dict(tau=(1.0, 0.8), G=-2.0)] * 4, precision="fp32", kernel=kernel)
        sim.set_geometry(np.repeat(t[None], 4, 0))
        sim.set_fields(np.repeat(r1[None], 4, 0), np.repeat(r2[None], 4, 0), np.repeat(u[None], 4, 0))
        done, res = lbm.lbm_run_to_steady(sim.ctx, 50, 1e-5, 3000, 4)
        out.append((done, res.copy(), sim.get_fields()))
        sim.close()
    assert out[0][0] == out[1][0] and np.array_equal(out[0][1], out[1][1])
    assert all(np.array_equal(x, y) for x, y in zip(out[0][2], out[1][2]))


def test_refusals(lbm):
    sim = lbm.Sim(8, 8, 8, [dict(tau=(1.0, 1.0), slip=0.5)], precision="fp32")
    sim.set_geometry(np.zeros((1, 8, 8, 8), np.uint8))
    with pytest.raises(lbm.LbmError):
        lbm.lbm_set_kernel(sim.ctx, lbm.KERNELS["persistent"])
    sim.close()
    sim = lbm.Sim(8, 8, 8, [dict(tau=(1.0, 1.0))], precision="fp32", kernel="persistent")
    sim.set_geometry(np.zeros((1, 8, 8, 8), np.uint8))
    with pytest.raises(lbm.LbmError):
        sim.set_params([dict(tau=(1.0, 1.0), slip=0.5)])
    sim.close()


def test_barrier_gives_up_and_context_recovers(lbm):
    """A barrier waiting for one arrival too many gives up after its bound
    (2e7 cycles, about 10 ms); LBM_ERR_TIMEOUT at the next reduction; with
    normal barriers the same context then updates as the compact path."""
    shape = (16, 12, 10)
    geo = [_geometry(shape, 0.2, 5)]
    p = [dict(tau=(0.8, 1.2), G=-1.8, rho_s=0.1)]
    sim = lbm.Sim(*shape, p, precision="fp32", kernel="persistent")
    sim.set_geometry(geo[0][0][None])
    sim.set_fields(geo[0][1][None], geo[0][2][None], geo[0][3][None])
    lbm.lbm_set_barrier_test(sim.ctx, 20_000_000, 1)
    t0 = time.perf_counter()
    sim.step(3)
    with pytest.raises(lbm.LbmError) as e:
        sim.reduce()
    assert e.value.status == 5 and "barrier" in str(e.value)
    assert time.perf_counter() - t0 < 30.0
    lbm.lbm_set_barrier_test(sim.ctx, 4_000_000_000, 0)
    sim.set_fields(geo[0][1][None], geo[0][2][None], geo[0][3][None])
    sim.step(5)
    a = sim.get_fields()
    sim.close()
    b = _run(lbm, "compact", shape, p, geo, [5], "fp32")[0]
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_batched_small_instances_timing(lbm):
    """16 instances of the 4 x 128 x 4 layered channel (the batched viscosity
    sweep) and 16 instances of 32^3: time per update of the two-launch compact
    update and of the persistent one (printed)."""
    import torch
    rows = []
    for shape, B, prec in (((4, 128, 4), 16, "fp32"), ((32, 32, 32), 16, "fp32"), ((16, 16, 16), 1, "fp32"),
                           ((4, 128, 4), 16, "fp64"), ((16, 16, 16), 1, "fp64")):
        t, r1, r2, u = W.layered_channel(*shape, layout="121") if shape[1] == 128 else W.droplet(*shape, shape[0] / 4)
        ms = {}
        for kernel in ("compact", "persistent"):
            sim = lbm.Sim(*shape, [dict(tau=(0.6, 1.5), G=-1.8, g=(1e-6, 0, 0))] * B, precision=prec,
                          kernel=kernel)
            sim.set_geometry(np.repeat(t[None], B, 0))
            sim.set_fields(np.repeat(r1[None], B, 0), np.repeat(r2[None], B, 0), np.repeat(u[None], B, 0))
            sim.step(200)
            torch.cuda.synchronize()
            a = time.perf_counter()
            sim.step(2000)
            sim.reduce()
            ms[kernel] = (time.perf_counter() - a) / 2000 * 1e3
            sim.close()
        rows.append((shape, B, prec, ms))
    print("ms per update:", rows)
