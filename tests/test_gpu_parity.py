"""GPU path vs the FP64 oracle, through the C ABI.

Tolerances (relative to the field's scale, max over cells):
  FP64 storage + FP64 arithmetic   1e-11  (after the whole run)
  FP32                              1e-5 on the densities and on u_F (5e-5 on the
                                    droplet's u_F, see DROPLET_BOUNDS)
  FP16 / BF16 shifted storage       densities 1e-3 / 6e-3, u_F 1e-2 / 6e-2 on the
                                    32^3 droplet after 1000 updates (rounding of the
                                    stored deviation: FP16 keeps 11 significant
                                    bits, BF16 8).  The velocity bound is looser:
                                    the storage leaves an absolute velocity error of
                                    ~2e-5 (FP16), set while the sharp initial
                                    interface drives |u_F| ~ 0.2, against a final
                                    spurious current of ~7e-3.
"""
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


def _rel(a, b):
    scale = max(np.abs(b).max(), 1e-30)
    return float(np.abs(a - b).max() / scale)


def _pair(lbm, oracle_mod, shape, params, t, r1, r2, u, steps, precision="fp64", eq_order=0, wall_model=0,
          kernel="auto"):
    nx, ny, nz = shape
    B = len(params)
    sim = lbm.Sim(nx, ny, nz, params, precision=precision, eq_order=eq_order, wall_model=wall_model,
                  kernel=kernel)
    sim.set_geometry(t.reshape((B, nz, ny, nx)))
    sim.set_fields(r1, r2, u)
    sim.step(steps)
    g = sim.get_fields()
    ref = oracle_mod.OracleSim(nx, ny, nz, params, eq_order=eq_order, wall_model=wall_model)
    ref.set_geometry(t.reshape((B, nz, ny, nx)))
    ref.set_fields(r1.reshape((B, nz, ny, nx)), r2.reshape((B, nz, ny, nx)), u.reshape((B, nz, ny, nx, 3)))
    ref.step(steps)
    o = ref.get_fields()
    return sim, ref, g, o


def _errs(g, o):
    return _rel(g[0], o[0]), _rel(g[1], o[1]), _rel(g[2], o[2])


KERNELS = ["two_pass", "fused", "cluster", "compact"]


@pytest.mark.parametrize("kernel", KERNELS)
def test_fp64_droplet_32cubed(lbm, oracle_mod, kernel):
    """32^3 periodic droplet, R = 8, G = -2.2, tau = 1, 1000 updates, FP64."""
    t, r1, r2, u = W.droplet(32, 32, 32, 8.0)
    p = [dict(tau=(1.0, 1.0), G=-2.2)]
    sim, ref, g, o = _pair(lbm, oracle_mod, (32, 32, 32), p, t, r1, r2, u, 1000, kernel=kernel)
    e = _errs(g, o)
    assert max(e) < 1e-11, e
    red = sim.reduce()[0]
    rref = ref.reduce()[0]
    assert abs(red[0] - rref[0]) / rref[0] < 1e-12 and abs(red[1] - rref[1]) / rref[1] < 1e-12


def _random_geometry(shape, frac, seed, inlet_outlet=False, lo=0.05, hi=1.0):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    t = np.where(rng.random((nz, ny, nx)) < frac, W.SOLID, W.FLUID).astype(np.uint8)
    if inlet_outlet:
        t[:, :, 0] = np.where(t[:, :, 0] == W.SOLID, W.SOLID, W.INLET)
        t[:, :, nx - 1] = np.where(t[:, :, nx - 1] == W.SOLID, W.SOLID, W.OUTLET)
    r1 = np.where(t == W.SOLID, 0.0, rng.uniform(lo, hi, t.shape))
    r2 = np.where(t == W.SOLID, 0.0, rng.uniform(lo, hi, t.shape))
    u = rng.uniform(-0.02, 0.02, t.shape + (3,))
    u[t == W.SOLID] = 0
    return t, r1, r2, u


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("shape", [(6, 5, 7), (13, 7, 9), (33, 3, 2), (70, 19, 23)])
@pytest.mark.parametrize("eq_order,wall_model", [(0, 0), (1, 1), (0, 1), (0, 2), (1, 2), (1, 3)])
def test_fp64_odd_grids_with_walls(lbm, oracle_mod, shape, eq_order, wall_model, kernel):
    """Odd grids (ragged tiles), random SOLID cells, wetting walls, extreme tau:
    cell by cell."""
    t, r1, r2, u = _random_geometry(shape, 0.2, 5 + sum(shape), lo=0.3, hi=0.7)
    p = [dict(tau=(0.5051, 5.6), G=-1.2, rho_s=0.3, g=(1e-4, -2e-5, 3e-5))]
    _, _, g, o = _pair(lbm, oracle_mod, shape, p, t[None], r1[None], r2[None], u[None], 20, eq_order=eq_order,
                       wall_model=wall_model, kernel=kernel)
    e = _errs(g, o)
    assert max(e) < 1e-12, e


@pytest.mark.parametrize("kernel", KERNELS)
def test_fp64_inlet_outlet(lbm, oracle_mod, kernel):
    shape = (12, 6, 5)
    t, r1, r2, u = _random_geometry(shape, 0.1, 9, inlet_outlet=True, lo=0.4, hi=0.6)
    p = [dict(tau=(0.6, 2.0), G=-1.0, rho_s=-0.2, rho_in=(0.1, 0.9), u_in=(0.01, 0.0, 0.0))]
    _, _, g, o = _pair(lbm, oracle_mod, shape, p, t[None], r1[None], r2[None], u[None], 30, kernel=kernel)
    e = _errs(g, o)
    assert max(e) < 1e-12, e


@pytest.mark.parametrize("tile,zchunk", [(0, 8), (1, 5), (2, 16), (3, 3)])
def test_fp64_fused_tilings(lbm, oracle_mod, tile, zchunk):
    """Every fused tiling, several z chunks and ragged edges, against the oracle."""
    shape = (45, 21, 19)
    t, r1, r2, u = _random_geometry(shape, 0.15, 77, lo=0.3, hi=0.7)
    p = [dict(tau=(0.7, 1.9), G=-1.4, rho_s=0.2, g=(2e-5, 0, 1e-5))]
    nx, ny, nz = shape
    sim = lbm.Sim(nx, ny, nz, p, kernel="fused")
    lbm.lbm_set_tiling(sim.ctx, tile, zchunk)
    sim.set_geometry(t[None])
    sim.set_fields(r1[None], r2[None], u[None])
    sim.step(12)
    ref = oracle_mod.OracleSim(nx, ny, nz, p)
    ref.set_geometry(t[None])
    ref.set_fields(r1[None], r2[None], u[None])
    ref.step(12)
    e = _errs(sim.get_fields(), ref.get_fields())
    assert max(e) < 1e-12, e


@pytest.mark.parametrize("kernel", KERNELS)
def test_fp64_batched_instances(lbm, oracle_mod, kernel):
    """Three instances with different parameters in one context."""
    shape = (8, 10, 6)
    geo = [_random_geometry(shape, 0.15, 20 + k, lo=0.3, hi=0.7) for k in range(3)]
    t = np.stack([x[0] for x in geo])
    r1 = np.stack([x[1] for x in geo])
    r2 = np.stack([x[2] for x in geo])
    u = np.stack([x[3] for x in geo])
    p = [dict(tau=(1.0, 1.0), G=-2.2), dict(tau=(0.52, 3.0), G=-1.7, rho_s=0.4, g=(0, 1e-4, 0)),
         dict(tau=(2.0, 0.6), G=-2.4, rho_s=-0.3, g=(1e-5, 0, 2e-5))]
    _, _, g, o = _pair(lbm, oracle_mod, shape, p, t, r1, r2, u, 25, kernel=kernel)
    assert max(_errs(g, o)) < 1e-12


# (densities, u_F) bounds per storage.  The periodic droplet has no preferred
# position: rounding noise moves it by a random walk over the 1000 updates, so
# its velocity field (a spurious current of ~7e-3) differs from the oracle's by
# an amount set by the rounding sequence (FP32: 7.9e-6 on the dense layout,
# 2.4e-5 with the packed-pair arithmetic of the compact layout).  The wall case
# has no such neutral mode and holds FP32 to 1e-5 and FP16 to 1e-3 on u_F.
DROPLET_BOUNDS = {"fp32": (1e-5, 5e-5), "fp16s": (1e-3, 1e-2), "bf16s": (6e-3, 6e-2)}
WALL_BOUNDS = {"fp32": (1e-5, 1e-5), "fp16s": (1e-3, 1e-3), "bf16s": (1e-2, 1e-2)}


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", ["fp32", "fp16s", "bf16s"])
def test_reduced_precision_droplet(lbm, oracle_mod, precision, kernel):
    """32^3 droplet, 1000 updates: FP32 arithmetic with FP32 / 16-bit storage;
    densities and u_F against the oracle within the storage's bounds."""
    t, r1, r2, u = W.droplet(32, 32, 32, 8.0)
    p = [dict(tau=(1.0, 1.0), G=-2.2)]
    _, _, g, o = _pair(lbm, oracle_mod, (32, 32, 32), p, t, r1, r2, u, 1000, precision=precision, kernel=kernel)
    e = _errs(g, o)
    rb, ub = DROPLET_BOUNDS[precision]
    assert e[0] < rb and e[1] < rb and e[2] < ub, e


@pytest.mark.parametrize("kernel", ["two_pass", "compact"])
@pytest.mark.parametrize("precision", ["fp32", "fp16s", "bf16s"])
def test_reduced_precision_walls(lbm, oracle_mod, precision, kernel):
    """Random walls, wetting wall potential and a body force, 20 updates:
    densities and u_F within the storage's bounds."""
    shape = (13, 7, 9)
    t, r1, r2, u = _random_geometry(shape, 0.2, 31, lo=0.3, hi=0.7)
    p = [dict(tau=(0.7, 1.5), G=-1.8, rho_s=0.3, g=(1e-4, 0, 0))]
    _, _, g, o = _pair(lbm, oracle_mod, shape, p, t[None], r1[None], r2[None], u[None], 20, precision=precision,
                       kernel=kernel)
    e = _errs(g, o)
    rb, ub = WALL_BOUNDS[precision]
    assert e[0] < rb and e[1] < rb and e[2] < ub, e


# absolute u_F bounds of the balanced walls (model 3) case below
WALL3_U_ABS = {"fp32": 1e-7, "fp16s": 2e-5, "bf16s": 1.5e-4}


@pytest.mark.parametrize("kernel", ["two_pass", "compact"])
@pytest.mark.parametrize("precision", ["fp32", "fp16s", "bf16s"])
def test_reduced_precision_walls_model3(lbm, oracle_mod, precision, kernel):
    """The wall case above with wall model 3.  Its walls move no momentum
    into the mixture, so the velocity field is only the decaying initial one
    (max |u_F| 3.6e-3 after 20 updates, against 4.5e-2 with model 0's vacuum
    walls) and a bound relative to it would measure the storage's absolute
    velocity error (about 1e-5 for FP16 whatever the flow) against a small
    field.  The densities keep the relative bounds; u_F is held to absolute
    bounds (measured FP16 1.1e-5, BF16 8.6e-5)."""
    shape = (13, 7, 9)
    t, r1, r2, u = _random_geometry(shape, 0.2, 31, lo=0.3, hi=0.7)
    p = [dict(tau=(0.7, 1.5), G=-1.8, rho_s=0.3, g=(1e-4, 0, 0))]
    _, _, g, o = _pair(lbm, oracle_mod, shape, p, t[None], r1[None], r2[None], u[None], 20, precision=precision,
                       kernel=kernel, wall_model=3)
    e = _errs(g, o)
    rb, _ = WALL_BOUNDS[precision]
    du = float(np.abs(g[2] - o[2]).max())
    assert e[0] < rb and e[1] < rb and du < WALL3_U_ABS[precision], (e, du)


def test_reductions_match_oracle(lbm, oracle_mod):
    shape = (16, 12, 10)
    t, r1, r2, u = _random_geometry(shape, 0.1, 41, lo=0.3, hi=0.7)
    p = [dict(tau=(0.8, 1.2), G=-2.0, g=(1e-4, 0, 0))]
    sim, ref, _, _ = _pair(lbm, oracle_mod, shape, p, t[None], r1[None], r2[None], u[None], 15)
    a = sim.reduce()[0]
    b = ref.reduce()[0]
    assert np.allclose(a[:2], b[:2], rtol=1e-13)
    assert np.allclose(a[2:5], b[2:5], rtol=1e-10, atol=1e-14)
    assert abs(a[5] - b[5]) <= 1e-10 * abs(b[5]) and abs(a[6] - b[6]) <= 1e-12
    sim.step(5)
    ref.step(5)
    a = sim.reduce()[0]
    b = ref.reduce()[0]
    assert abs(a[5] - b[5]) <= 1e-9 * abs(b[5])


def test_fp32_reductions_against_fp64_sums(lbm):
    """With FP32 fields the reduction forms each cell's terms in FP32 and
    sums groups of eight cells in FP32 before FP64: masses, momentum,
    max |u_F| and the residual against FP64 sums of the exported fields."""
    shape = (40, 30, 20)
    t, r1, r2, u = _random_geometry(shape, 0.2, 43, lo=0.3, hi=0.7)
    sim = lbm.Sim(*shape, [dict(tau=(0.8, 1.3), G=-2.0, rho_s=0.2, g=(1e-4, 0, 0))], precision="fp32")
    sim.set_geometry(t[None])
    sim.set_fields(r1[None], r2[None], u[None])
    sim.step(10)
    sim.reduce()
    _, _, u0 = sim.get_fields()
    sim.step(7)
    red = sim.reduce()[0]
    a, b, v = sim.get_fields()
    fl = (t != W.SOLID)[None]
    rho = a + b
    assert abs(red[0] - a[fl].sum()) < 1e-6 * a[fl].sum() and abs(red[1] - b[fl].sum()) < 1e-6 * b[fl].sum()
    P = (rho[..., None] * v)[fl].sum(axis=0)
    scale = np.abs(rho[..., None] * v)[fl].sum()
    assert np.all(np.abs(red[2:5] - P) < 1e-6 * scale), (red[2:5], P)
    d2 = ((v - u0) ** 2)[fl].sum()
    u2 = (v ** 2)[fl].sum()
    res = np.sqrt(d2) / (7 * np.sqrt(u2))
    assert abs(red[5] - res) < 1e-4 * res, (red[5], res)
    umax = np.sqrt((v ** 2).sum(-1))[fl].max()
    assert abs(red[6] - umax) < 1e-6 * umax, (red[6], umax)


def test_reductions_are_deterministic(lbm):
    t, r1, r2, u = W.droplet(24, 24, 24, 6.0)
    outs = []
    for _ in range(2):
        sim = lbm.Sim(24, 24, 24, [dict(tau=(1.0, 0.7), G=-2.2)], precision="fp32")
        sim.set_geometry(t[None])
        sim.set_fields(r1[None], r2[None], u[None])
        sim.step(50)
        outs.append(sim.reduce())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("kernel", ["auto", "compact"])
def test_checkpoint_roundtrip_bitwise(lbm, kernel):
    t, r1, r2, u = _random_geometry((10, 9, 8), 0.1, 51, lo=0.3, hi=0.7)
    p = [dict(tau=(0.9, 1.4), G=-2.0, rho_s=0.1, g=(1e-5, 0, 0))]
    for prec in ("fp64", "fp16s"):
        a = lbm.Sim(10, 9, 8, p, precision=prec, kernel=kernel)
        a.set_geometry(t[None])
        a.set_fields(r1[None], r2[None], u[None])
        a.step(10)
        st = a.get_state()
        a.step(10)
        fa = a.get_fields()
        b = lbm.Sim(10, 9, 8, p, precision=prec, kernel=kernel)
        b.set_state(st)
        b.step(10)
        fb = b.get_fields()
        for x, y in zip(fa, fb):
            assert np.array_equal(x, y)


def test_errors_reported(lbm):
    sim = lbm.Sim(4, 4, 4, [dict(tau=(1.0, 1.0))])
    with pytest.raises(lbm.LbmError) as e:
        sim.step(1)
    assert e.value.status == 6
    with pytest.raises(lbm.LbmError) as e:
        sim.set_geometry(np.full((1, 4, 4, 4), 7, np.uint8))
    assert e.value.status == 1
    with pytest.raises(lbm.LbmError) as e:
        sim.set_geometry(np.full((1, 4, 4, 4), 1, np.uint8))
    assert e.value.status == 1


def test_divergence_is_flagged(lbm):
    """A blow-up (tau -> 1/2 with a huge body force) is reported as
    LBM_ERR_DIVERGED by the reduction, and the context stays usable."""
    t, r1, r2, u = W.droplet(8, 8, 8, 2.0)
    sim = lbm.Sim(8, 8, 8, [dict(tau=(0.5001, 0.5001), G=-2.2, g=(0.5, 0.3, 0.0))], precision="fp32")
    sim.set_geometry(t[None])
    sim.set_fields(r1[None], r2[None], u[None])
    sim.step(200)
    with pytest.raises(lbm.LbmError) as e:
        sim.reduce()
    assert e.value.status == 4
    sim.get_fields()


@pytest.mark.parametrize("kernel", ["auto", "compact"])
def test_distributions_roundtrip(lbm, oracle_mod, kernel):
    """FP64 distributions exported by the library step identically in the oracle."""
    shape = (9, 8, 7)
    t, r1, r2, u = _random_geometry(shape, 0.1, 61, lo=0.3, hi=0.7)
    p = [dict(tau=(0.8, 1.1), G=-2.0, rho_s=0.2)]
    sim = lbm.Sim(*shape, p, kernel=kernel)
    sim.set_geometry(t[None])
    sim.set_fields(r1[None], r2[None], u[None])
    sim.step(7)
    f = sim.get_f()
    ref = oracle_mod.OracleSim(*shape, p)
    ref.set_geometry(t[None])
    ref.set_fields(r1[None], r2[None], u[None])
    ref.set_f(f)
    ref.step(1)
    sim.step(1)
    assert max(_errs(sim.get_fields(), ref.get_fields())) < 1e-13
    sim.set_f(f)
    sim.step(1)
    assert max(_errs(sim.get_fields(), ref.get_fields())) < 1e-13
    assert np.all(f[:, :, :, t == W.SOLID] == 0.0)  # SOLID cells carry no distributions


LAYOUT_BOUND = {"fp32": 1e-5, "fp16s": 1e-3, "bf16s": 6e-3}


def _layout_case(lbm, precision, kernel):
    shape = (37, 21, 11)
    t, r1, r2, u = _random_geometry(shape, 0.3, 71, lo=0.3, hi=0.7)
    p = [dict(tau=(0.8, 1.3), G=-1.9, rho_s=-0.2, g=(2e-5, 1e-5, 0)),
         dict(tau=(1.1, 0.6), G=-2.1, rho_s=0.3, g=(0, 0, 3e-5))]
    t2 = np.stack([t, np.roll(t, 5, axis=2)])
    r1s, r2s, us = np.stack([r1, np.roll(r1, 5, axis=2)]), np.stack([r2, np.roll(r2, 5, axis=2)]), np.stack([u, u])
    s_ = lbm.Sim(*shape, p, precision=precision, kernel=kernel)
    s_.set_geometry(t2)
    s_.set_fields(r1s, r2s, us)
    return s_


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s", "bf16s"])
def test_layouts_agree(lbm, precision):
    """A run that switches between the compact and the dense strategy every
    few updates (converting the layout each time) against a dense-only run.
    FP64 runs the same scalar arithmetic in both layouts and ends bitwise
    equal, fields and distributions.  The FP32-arithmetic storages run the
    compact update on packed FP32 pairs, rounded in another order, so there
    the two agree within the precision's parity bound."""
    dense = _layout_case(lbm, precision, "two_pass")
    mixed = _layout_case(lbm, precision, "compact")
    for rnd in range(4):
        dense.step(3)
        lbm.lbm_set_kernel(mixed.ctx, "compact" if rnd % 2 == 0 else "two_pass")
        mixed.step(3)
    lbm.lbm_set_kernel(mixed.ctx, "compact")
    mixed.step(2)
    dense.step(2)
    if precision == "fp64":
        for x, y in zip(dense.get_fields(), mixed.get_fields()):
            assert np.array_equal(x, y)
        assert np.array_equal(dense.get_f(), mixed.get_f())
    else:
        g, o = mixed.get_fields(), dense.get_fields()
        e = _errs(g, o)
        assert _rel(g[0], o[0]) < LAYOUT_BOUND[precision] and _rel(g[1], o[1]) < LAYOUT_BOUND[precision], e


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s", "bf16s"])
def test_layout_conversion_is_exact(lbm, precision):
    """Converting the state between the compact and the dense layout changes
    no bit: compact updates interrupted by reads of f (each converts to the
    dense layout, the next update back) end bitwise equal to the same
    updates run without interruption."""
    straight = _layout_case(lbm, precision, "compact")
    broken = _layout_case(lbm, precision, "compact")
    straight.step(6)
    for _ in range(3):
        broken.step(2)
        broken.get_f()
    for x, y in zip(straight.get_fields(), broken.get_fields()):
        assert np.array_equal(x, y)
    assert np.array_equal(straight.get_f(), broken.get_f())


# ------------------------------------------------------------------ batched persistent launch (sweeps)

# With both components at nu = 0.0017 (tau = 0.5051) the layered channel is
# unstable at G = -2.2 (also in the oracle, from sharp or relaxed layers) and
# stable at G = -1.8, so the sweep uses G = -1.8.
SWEEP_G = -1.8


def _poiseuille_sweep():
    """Two-layer channel sweep (4 x 128 x 4, walls at y): viscosity ratio
    {1, 10, 100, 1000} with minimum nu = 0.0017, the low-viscosity component
    along the walls or in the core, layouts 1|2|1 and 1|2: 16 instances."""
    cases = []
    for ratio in (1, 10, 100, 1000):
        for low_at_wall in (True, False):
            for layout in ("121", "12"):
                lo, hi = 0.0017, 0.0017 * ratio
                nu1, nu2 = (lo, hi) if low_at_wall else (hi, lo)
                cases.append((layout, nu1, nu2))
    return cases


@pytest.mark.parametrize("kernel", ["cluster", "fused"])
def test_fp64_batched_sweep_matches_oracle(lbm, oracle_mod, kernel):
    """All 16 instances of the sweep in one context, 2000 updates in one call
    (one persistent launch with the cluster kernel), against the oracle."""
    cases = _poiseuille_sweep()
    ts, r1s, r2s, us, ps = [], [], [], [], []
    for layout, nu1, nu2 in cases:
        t, r1, r2, u = W.layered_channel(4, 128, 4, layout=layout, wall_comp_nu=nu1, core_comp_nu=nu2, g=4e-8)
        ts.append(t), r1s.append(r1), r2s.append(r2), us.append(u)
        ps.append(dict(tau=(nu1 * 3 + 0.5, nu2 * 3 + 0.5), G=SWEEP_G, g=(4e-8, 0, 0)))
    t, r1, r2, u = np.stack(ts), np.stack(r1s), np.stack(r2s), np.stack(us)
    sim = lbm.Sim(4, 128, 4, ps, kernel=kernel)
    sim.set_geometry(t)
    sim.set_fields(r1, r2, u)
    l0 = sim.launches
    sim.step(2000)
    if kernel == "cluster":
        assert sim.launches - l0 == 1
    g = sim.get_fields()
    ref = oracle_mod.OracleSim(4, 128, 4, ps)
    ref.set_geometry(t)
    ref.set_fields(r1, r2, u)
    ref.step(2000)
    o = ref.get_fields()
    for b in range(len(ps)):
        e = _errs([x[b] for x in g], [x[b] for x in o])
        assert max(e) < 1e-11, (b, e)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_sweep_analytic_profile(lbm, precision):
    """The 16-instance sweep on relaxed layers, 20k updates in one launch:
    each profile stays on the steady solution with the density-weighted
    viscosity (2 % for 1|2|1, 6 % for 1|2, as for the oracle)."""
    import sys
    sys.path.insert(0, __file__.rsplit("/", 1)[0])
    from tests import analytic
    cases = _poiseuille_sweep()
    g = 4e-8
    ts, r1s, r2s, us, p0, p1 = [], [], [], [], [], []
    for layout, nu1, nu2 in cases:
        t, r1, r2, u = W.layered_channel(4, 128, 4, layout=layout, analytic_velocity=False)
        ts.append(t), r1s.append(r1), r2s.append(r2), us.append(u)
        p0.append(dict(tau=(nu1 * 3 + 0.5, nu2 * 3 + 0.5), G=SWEEP_G))
        p1.append(dict(tau=(nu1 * 3 + 0.5, nu2 * 3 + 0.5), G=SWEEP_G, g=(g, 0, 0)))
    t = np.stack(ts)
    relax = lbm.Sim(4, 128, 4, p0, precision=precision)
    relax.set_geometry(t)
    relax.set_fields(np.stack(r1s), np.stack(r2s), np.stack(us))
    relax.step(30000)
    a, b, _ = relax.get_fields()

    def integral(a, b, nu1, nu2):
        a1, b1 = a[0, 1:-1, 0], b[0, 1:-1, 0]
        rho = a1 + b1
        p = np.clip(a1 / rho, 0, 1)
        return analytic.layered_poiseuille(rho, p * nu1 + (1 - p) * nu2, g)

    u0 = np.zeros(a.shape + (3,))
    for k, (layout, nu1, nu2) in enumerate(cases):
        u0[k, :, 1:-1, :, 0] = integral(a[k], b[k], nu1, nu2)[None, :, None]
    run = lbm.Sim(4, 128, 4, p1, precision=precision)
    run.set_geometry(t)
    run.set_fields(a, b, u0)
    run.step(20000)
    a2, b2, v = run.get_fields()
    for k, (layout, nu1, nu2) in enumerate(cases):
        ref = integral(a2[k], b2[k], nu1, nu2)
        ux = v[k, 0, 1:-1, 0, 0]
        tol = 0.02 if layout == "121" else 0.06
        err = np.abs(ux - ref).max() / np.abs(ref).max()
        assert np.isfinite(err) and err < tol, (k, layout, nu1, nu2, err)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp16s", 1e-3)])
def test_benchmark_workload_full_size(lbm, oracle_mod, precision, tol):
    """The benchmark's own configuration: 256^3 packed spheres, AUTO kernel
    (compact layout), every cell against the oracle after 3 updates."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    t, r1, r2, u = bench.workload(256, "spheres")
    _, _, g, o = _pair(lbm, oracle_mod, (256, 256, 256), [bench.PARAMS], t[None], r1[None], r2[None], u[None], 3,
                       precision=precision, wall_model=2)
    e = _errs(g, o)
    assert max(e) < tol, e


@pytest.mark.parametrize("kernel", ["two_pass", "compact", "fused"])
@pytest.mark.parametrize("shape", [(1, 9, 7), (5, 1, 3), (4, 6, 1), (1, 1, 8)])
def test_fp64_degenerate_axes(lbm, oracle_mod, shape, kernel):
    """Axes of length 1 (the neighbour along that axis is the cell itself):
    cell by cell against the oracle, with walls."""
    t, r1, r2, u = _random_geometry(shape, 0.15, 91 + sum(shape), lo=0.3, hi=0.7)
    if not (t == W.FLUID).any():
        t.flat[0] = W.FLUID
    r1[t == W.SOLID] = 0
    r2[t == W.SOLID] = 0
    p = [dict(tau=(0.8, 1.3), G=-1.6, rho_s=0.2, g=(1e-4, 0, 2e-5))]
    _, _, g, o = _pair(lbm, oracle_mod, shape, p, t[None], r1[None], r2[None], u[None], 15, wall_model=2,
                       kernel=kernel)
    e = _errs(g, o)
    assert max(e) < 1e-12, e


def test_zero_updates_and_empty_steps(lbm, oracle_mod):
    """lbm_step(0) changes nothing and launches nothing."""
    t, r1, r2, u = _random_geometry((9, 8, 7), 0.2, 93, lo=0.3, hi=0.7)
    sim = lbm.Sim(9, 8, 7, [dict(tau=(0.9, 1.1), G=-1.8)])
    sim.set_geometry(t[None])
    sim.set_fields(r1[None], r2[None], u[None])
    f0 = sim.get_f()
    l0 = sim.launches
    sim.step(0)
    assert sim.launches == l0
    assert np.array_equal(sim.get_f(), f0)


def test_compact_limits_fall_back(lbm):
    """Beyond the compact layout's coordinate limits AUTO runs the dense
    two-pass update and an explicit request for COMPACT is refused."""
    sim = lbm.Sim(2049, 4, 4, [dict(tau=(1.0, 1.0), G=-1.8)], precision="fp32")
    t = np.zeros((1, 4, 4, 2049), np.uint8)
    sim.set_geometry(t)
    assert lbm.lbm_resolved_kernel(sim.ctx, 10) == "two_pass"
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_kernel(sim.ctx, "compact")
    assert e.value.status == 1
    small = lbm.Sim(64, 64, 16, [dict(tau=(1.0, 1.0), G=-1.8)], precision="fp32")
    small.set_geometry(np.zeros((1, 16, 64, 64), np.uint8))
    # up to 65,536 non-solid cells AUTO steps n >= 8 updates in one persistent launch
    assert lbm.lbm_resolved_kernel(small.ctx, 10) == "persistent"
    assert lbm.lbm_resolved_kernel(small.ctx, 1) == "compact"
    larger = lbm.Sim(64, 64, 17, [dict(tau=(1.0, 1.0), G=-1.8)], precision="fp32")
    larger.set_geometry(np.zeros((1, 17, 64, 64), np.uint8))
    assert lbm.lbm_resolved_kernel(larger.ctx, 10) == "compact"


@pytest.mark.parametrize("precision,bound", [("fp32", 1e-6), ("fp16s", 5e-5), ("bf16s", 5e-3)])
def test_reduced_precision_mass_conservation(lbm, precision, bound):
    """Per-component mass over 1000 updates of the 32^3 droplet (the update
    conserves it exactly; what drifts is storage rounding).  The FP16 bound
    needs the 2^12 scale of the stored deviations: unscaled, the bulk's tiny
    deviations sit in FP16's subnormal range."""
    t, r1, r2, u = W.droplet(32, 32, 32, 8.0)
    sim = lbm.Sim(32, 32, 32, [dict(tau=(1.0, 1.0), G=-2.2)], precision=precision, kernel="compact")
    sim.set_geometry(t[None])
    sim.set_fields(r1[None], r2[None], u[None])
    m0 = sim.reduce()[0][:2].copy()
    sim.step(1000)
    m1 = sim.reduce()[0][:2]
    assert np.all(np.abs(m1 - m0) / m0 < bound), (m0, m1)


# ---------------------------------------------------------------- rough channel crop (benchmark's rough channel)

def _rough_crop():
    import bench
    t, r1, r2, u = W.rough_channel(64, 32, 32, seed=4, invaded_length=8, ends="periodic")
    return t, r1, r2, u, [bench.ROUGH_PARAMS]


@pytest.mark.parametrize("kernel", ["compact", "two_pass"])
def test_rough_channel_crop_fp64(lbm, oracle_mod, kernel):
    """The rough channel's recipe at 64 x 32 x 32 (walls with bumps, an invading
    slug at nu = 0.0017 against nu = 1.7, wetting walls, body force), FP64,
    1000 updates: cell by cell against the oracle, and both conserve each
    component's mass to 1e-12."""
    t, r1, r2, u, p = _rough_crop()
    sim, ref, g, o = _pair(lbm, oracle_mod, (64, 32, 32), p, t[None], r1[None], r2[None], u[None], 1000,
                           wall_model=2, kernel=kernel)
    assert max(_errs(g, o)) < 1e-11
    m0 = np.array([r1[t != W.SOLID].sum(), r2[t != W.SOLID].sum()])
    for red in (sim.reduce()[0], ref.reduce()[0]):
        assert np.all(np.abs(red[:2] - m0) / m0 < 1e-12)


# per storage: densities, u_F, per-component mass drift over the 1000 updates
ROUGH_BOUNDS = {"fp32": (1e-5, 1e-5, 1e-7), "fp16s": (1e-3, 5e-3, 2e-5), "bf16s": (6e-3, 3e-2, 5e-4)}


@pytest.mark.parametrize("precision", ["fp32", "fp16s", "bf16s"])
def test_rough_channel_crop_storage(lbm, oracle_mod, precision):
    """The same crop in the FP32-arithmetic storages against the FP64 oracle
    after 1000 updates: fields within the storage's bounds, mass drift of the
    storage rounding within its bound (the update itself conserves mass)."""
    t, r1, r2, u, p = _rough_crop()
    sim, _, g, o = _pair(lbm, oracle_mod, (64, 32, 32), p, t[None], r1[None], r2[None], u[None], 1000,
                         precision=precision, wall_model=2)
    e = _errs(g, o)
    rb, ub, mb = ROUGH_BOUNDS[precision]
    assert e[0] < rb and e[1] < rb and e[2] < ub, e
    m0 = np.array([r1[t != W.SOLID].sum(), r2[t != W.SOLID].sum()])
    drift = np.abs(sim.reduce()[0][:2] - m0) / m0
    assert np.all(drift < mb), drift


# ---------------------------------------------------------------- Galilean invariance (eq_order 1)

@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_shear_wave_on_stream(lbm, oracle_mod, precision, tol):
    """A shear wave on a uniform stream with the full equilibrium: the GPU
    matches the oracle, whose wave decays at the rate of the wave at rest and
    moves with the stream (the oracle pin of Galilean invariance)."""
    nx = 32
    x = np.arange(nx) + 0.5
    k = 2 * np.pi / nx
    u = np.zeros((1, 1, 1, nx, 3))
    u[..., 0] = 0.05
    u[..., 1] = 1e-3 * np.sin(k * x)
    t = np.zeros((1, 1, 1, nx), np.uint8)
    r = np.full((1, 1, 1, nx), 0.5)
    _, _, g, o = _pair(lbm, oracle_mod, (nx, 1, 1), [dict(tau=(0.8, 0.8), G=0.0)], t, r, r, u, 200,
                       precision=precision, eq_order=1)
    assert max(_errs(g, o)) < tol
