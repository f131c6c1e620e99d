"""The single-read fused update on the compact layout (LBM_KERNEL_FUSED_COMPACT).

It evaluates the update of Eq. 9 with the same FP32 operations, in the same
order, as the compact two-pass update; only where f and psi are read from
differs (f pulled once, psi kept in shared memory).  So the two strategies must
agree bit for bit on every geometry: bands of rows that end inside the grid or
wrap around it, CTAs without rows, chunks of one plane, degenerate axes,
INLET/OUTLET planes, all wall models and both equilibrium orders, batches of
instances.  The oracle comparison then carries over; one case checks it
directly.
"""
import numpy as np
import pytest

from paper_1711_03254_gb300 import workloads as W
from tests.test_gpu_parity import _errs, _pair, _random_geometry

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


def _run(lbm, shape, params, t, r1, r2, u, steps, precision, kernel, eq_order=0, wall_model=2, chunks=(1,)):
    nx, ny, nz = shape
    B = len(params)
    sim = lbm.Sim(nx, ny, nz, params, precision=precision, eq_order=eq_order, wall_model=wall_model, kernel=kernel)
    sim.set_geometry(t.reshape((B, nz, ny, nx)))
    sim.set_fields(r1.reshape((B, nz, ny, nx)), r2.reshape((B, nz, ny, nx)), u.reshape((B, nz, ny, nx, 3)))
    resolved = lbm.lbm_resolved_kernel(sim.ctx, 1)
    done = 0
    for c in chunks:
        sim.step(c)
        done += c
    while done < steps:
        sim.step(min(7, steps - done))
        done += min(7, steps - done)
    out = (sim.get_f(), sim.get_fields(), sim.reduce(allow_diverged=True))
    sim.close()
    return resolved, out


def _same(lbm, shape, params, t, r1, r2, u, steps, precision, **kw):
    rf, (f1, g1, red1) = _run(lbm, shape, params, t, r1, r2, u, steps, precision, "fused_compact", **kw)
    rc, (f2, g2, red2) = _run(lbm, shape, params, t, r1, r2, u, steps, precision, "compact", **kw)
    assert rf == "fused_compact" and rc == "compact"
    assert np.isfinite(f2).all(), "the compared case must stay finite"
    np.testing.assert_array_equal(f1, f2)
    for x, y in zip(g1, g2):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(red1, red2)


@pytest.mark.parametrize("precision", ["fp16s", "bf16s", "fp32"])
@pytest.mark.parametrize("shape", [(13, 7, 9), (33, 21, 17), (40, 37, 5), (6, 16, 3), (9, 17, 2)])
@pytest.mark.parametrize("eq_order,wall_model", [(0, 2), (1, 0), (0, 1), (0, 3)])
def test_bitwise_equal_to_compact_two_pass(lbm, precision, shape, eq_order, wall_model):
    """Random walls, wetting wall potential, body force, extreme tau: every
    stored value, the fields and the reductions after 20 updates."""
    t, r1, r2, u = _random_geometry(shape, 0.2, 3 + sum(shape), lo=0.3, hi=0.7)
    p = [dict(tau=(0.5051, 5.6), G=-1.4, rho_s=0.3, g=(1e-4, -2e-5, 3e-5))]
    _same(lbm, shape, p, t[None], r1[None], r2[None], u[None], 20, precision, eq_order=eq_order,
          wall_model=wall_model)


@pytest.mark.parametrize("shape", [(1, 9, 7), (5, 1, 3), (4, 6, 1), (1, 1, 8), (7, 33, 1)])
def test_bitwise_degenerate_axes(lbm, shape):
    """Length-1 axes: the band's outside rows and the halo planes are the
    cells' own rows and planes."""
    t, r1, r2, u = _random_geometry(shape, 0.1, 11 + sum(shape), lo=0.3, hi=0.7)
    t.reshape(-1)[0] = W.FLUID
    r1.reshape(-1)[0] = 0.5
    r2.reshape(-1)[0] = 0.5
    p = [dict(tau=(0.7, 1.3), G=-1.6, rho_s=-0.2, g=(1e-5, 2e-5, -1e-5))]
    _same(lbm, shape, p, t[None], r1[None], r2[None], u[None], 15, "fp16s")


@pytest.mark.parametrize("precision", ["fp16s", "fp32"])
def test_bitwise_inlet_outlet(lbm, precision):
    shape = (24, 18, 11)
    t, r1, r2, u = _random_geometry(shape, 0.1, 9, inlet_outlet=True, lo=0.4, hi=0.6)
    p = [dict(tau=(0.6, 2.0), G=-1.0, rho_s=-0.2, rho_in=(0.1, 0.9), u_in=(0.01, 0.0, 0.0))]
    _same(lbm, shape, p, t[None], r1[None], r2[None], u[None], 30, precision)


def test_bitwise_batched_instances(lbm):
    """Instances of different geometry and parameters in one launch."""
    shape = (20, 35, 13)
    geo = [_random_geometry(shape, 0.1 + 0.1 * k, 20 + k, lo=0.3, hi=0.7) for k in range(3)]
    t = np.stack([x[0] for x in geo])
    r1 = np.stack([x[1] for x in geo])
    r2 = np.stack([x[2] for x in geo])
    u = np.stack([x[3] for x in geo])
    p = [dict(tau=(1.0, 1.0), G=-2.2), dict(tau=(0.52, 3.0), G=-1.7, rho_s=0.4, g=(0, 1e-4, 0)),
         dict(tau=(2.0, 0.6), G=-2.4, rho_s=-0.3, g=(1e-5, 0, 2e-5))]
    _same(lbm, shape, p, t, r1, r2, u, 25, "fp16s", chunks=(1, 2, 3))


def test_bitwise_droplet_all_fluid(lbm):
    """No SOLID cell: every row full, the lag buffer at its largest."""
    t, r1, r2, u = W.droplet(48, 40, 36, 9.0)
    _same(lbm, (48, 40, 36), [dict(tau=(1.0, 0.7), G=-2.2)], t[None], r1[None], r2[None], u[None], 50, "fp16s")


@pytest.mark.parametrize("precision", ["fp32", "fp16s", "bf16s"])
def test_droplet_against_oracle(lbm, oracle_mod, precision):
    """32^3 droplet, 1000 updates, against the FP64 oracle within the storage's
    bounds on the densities and u_F."""
    from tests.test_gpu_parity import DROPLET_BOUNDS
    t, r1, r2, u = W.droplet(32, 32, 32, 8.0)
    _, _, g, o = _pair(lbm, oracle_mod, (32, 32, 32), [dict(tau=(1.0, 1.0), G=-2.2)], t, r1, r2, u, 1000,
                       precision=precision, kernel="fused_compact")
    e = _errs(g, o)
    rb, ub = DROPLET_BOUNDS[precision]
    assert e[0] < rb and e[1] < rb and e[2] < ub, e


def test_benchmark_workload_bitwise(lbm):
    """The benchmark's 256^3 packed spheres, FP16 storage: the fused compact
    update equals the compact two-pass one after 3 updates."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    t, r1, r2, u = bench.workload(256, "spheres")
    _same(lbm, (256, 256, 256), [bench.PARAMS], t[None], r1[None], r2[None], u[None], 3, "fp16s")


def test_fp64_falls_back_and_set_kernel_refuses(lbm):
    """FP64 has no fused compact update: setting it is an argument error."""
    with pytest.raises(lbm.LbmError) as e:
        lbm.Sim(8, 8, 8, [dict(tau=(1.0, 1.0), G=-2.0)], precision="fp64", kernel="fused_compact")
    assert e.value.status == 1
