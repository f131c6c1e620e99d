"""Pins of the oracle's partial-slip walls (the surface scattering model of
Sec. 2 read as a blend: a wall bounces back the fraction 1 - slip of the
particles and reflects the fraction slip specularly about the voxel wall).

What the mathematics fixes:
  * slip = 0 is the bounce-back wall, unchanged;
  * every post-collision value that meets a wall is used exactly once, so each
    component's mass is conserved to rounding for any slip and geometry;
  * specular reflection keeps the momentum along a flat wall: with slip = 1 a
    uniform stream along the walls of a channel is an exact steady state, and
    a body force raises the momentum by exactly F per update (no wall
    friction), where the bounce-back wall brakes both;
  * the cube symmetries hold with slip as without.
"""
import numpy as np
import pytest

from paper_1711_03254_gb300 import workloads as W


def _random_walls(shape, seed, frac=0.25):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    t = np.where(rng.random((nz, ny, nx)) < frac, W.SOLID, W.FLUID).astype(np.uint8)
    r1 = np.where(t == W.SOLID, 0.0, rng.uniform(0.3, 0.7, t.shape))
    r2 = np.where(t == W.SOLID, 0.0, rng.uniform(0.3, 0.7, t.shape))
    u = rng.uniform(-0.03, 0.03, t.shape + (3,))
    u[t == W.SOLID] = 0
    return t, r1, r2, u


def _sim(oracle_mod, shape, p, t, r1, r2, u, wall_model=2):
    nx, ny, nz = shape
    sim = oracle_mod.OracleSim(nx, ny, nz, [p], wall_model=wall_model)
    sim.set_geometry(t[None])
    sim.set_fields(r1[None], r2[None], u[None])
    return sim


def test_no_slip_is_bounce_back(oracle_mod):
    shape = (9, 7, 6)
    t, r1, r2, u = _random_walls(shape, 3)
    p = dict(tau=(0.7, 1.3), G=-1.5, rho_s=0.2, g=(1e-4, 0, 0))
    a = _sim(oracle_mod, shape, p, t, r1, r2, u)
    b = _sim(oracle_mod, shape, dict(p, slip=0.0), t, r1, r2, u)
    a.step(15)
    b.step(15)
    assert np.array_equal(a.get_f(), b.get_f())


def _mass_drift(oracle_mod, slip, seed=4, steps=40):
    shape = (11, 9, 7)
    t, r1, r2, u = _random_walls(shape, seed)
    sim = _sim(oracle_mod, shape, dict(tau=(0.6, 1.7), G=-1.8, rho_s=0.3, slip=slip), t, r1, r2, u)
    m0 = sim.reduce()[0][:2].copy()
    sim.step(steps)
    m1 = sim.reduce()[0][:2]
    return float(np.max(np.abs(m1 - m0) / m0))


@pytest.mark.parametrize("slip", [0.3, 1.0])
def test_slip_conserves_mass(oracle_mod, slip):
    assert _mass_drift(oracle_mod, slip) < 1e-13


def _channel_stream(oracle_mod, slip, g=0.0, U=0.02, steps=200):
    """Channel 4 x 10 x 3 with SOLID rows y = 0 and 9, one fluid (50/50, no
    coupling) streaming along x at U; returns max |u_x - U(t)| over the fluid
    and the x momentum gained per update against the force per update."""
    nx, ny, nz = 4, 10, 3
    t = np.zeros((nz, ny, nx), np.uint8)
    t[:, 0, :] = W.SOLID
    t[:, ny - 1, :] = W.SOLID
    fluid = t != W.SOLID
    r = np.where(fluid, 0.5, 0.0)
    u = np.zeros(t.shape + (3,))
    u[fluid, 0] = U
    sim = _sim(oracle_mod, (nx, ny, nz), dict(tau=(0.8, 0.8), G=0.0, slip=slip, g=(g, 0, 0)), t, r, r, u)
    sim.step(1)  # (the reported momentum is that of u_F, half a force ahead once stepping)
    P0 = sim.reduce()[0][2]
    sim.step(steps)
    P1 = sim.reduce()[0][2]
    _, _, v = sim.get_fields()
    ux = v[0][..., 0][fluid]
    F = g * fluid.sum()  # total density 1 per fluid cell
    return float(np.abs(ux - ux.mean()).max()), (P1 - P0) / steps, F


def test_specular_wall_keeps_a_uniform_stream(oracle_mod):
    dev, _, _ = _channel_stream(oracle_mod, 1.0)
    assert dev < 1e-14
    dev_bb, _, _ = _channel_stream(oracle_mod, 0.0)
    assert dev_bb > 1e-4  # the bounce-back wall shears the stream


def test_specular_wall_has_no_friction(oracle_mod):
    _, dP, F = _channel_stream(oracle_mod, 1.0, g=1e-5, U=0.0)
    assert abs(dP - F) < 1e-12 * F
    _, dP_bb, _ = _channel_stream(oracle_mod, 0.0, g=1e-5, U=0.0)
    assert dP_bb < 0.99 * F


def test_poiseuille_flux_grows_with_slip(oracle_mod):
    flux = []
    for slip in (0.0, 0.25, 0.5, 0.75):
        nx, ny, nz = 1, 14, 1
        t = np.zeros((nz, ny, nx), np.uint8)
        t[:, 0, :] = W.SOLID
        t[:, ny - 1, :] = W.SOLID
        fl = t != W.SOLID
        r = np.where(fl, 0.5, 0.0)
        sim = _sim(oracle_mod, (nx, ny, nz), dict(tau=(0.8, 0.8), G=0.0, slip=slip, g=(1e-6, 0, 0)), t, r, r,
                   np.zeros(t.shape + (3,)))
        sim.step(3000)
        _, _, v = sim.get_fields()
        flux.append(float(v[0][..., 0][fl].sum()))
    assert all(b > a * 1.01 for a, b in zip(flux, flux[1:])), flux


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_slip_mirror_symmetry(oracle_mod, axis):
    """Reflecting the whole problem along an axis reflects the evolution."""
    shape = (7, 6, 5)
    t, r1, r2, u = _random_walls(shape, 9)
    g = np.array([2e-5, -1e-5, 3e-5])
    p = dict(tau=(0.7, 1.4), G=-1.6, rho_s=0.25, slip=0.6, g=tuple(g))
    ax = 2 - axis  # array axis of the lattice axis
    flip = lambda a: np.flip(a, axis=ax).copy()
    def flip_u(v):
        w = np.flip(v, axis=ax).copy()
        w[..., axis] *= -1
        return w
    gm = g.copy()
    gm[axis] *= -1
    a = _sim(oracle_mod, shape, p, t, r1, r2, u)
    b = _sim(oracle_mod, shape, dict(p, g=tuple(gm)), flip(t), flip(r1), flip(r2), flip_u(u))
    a.step(20)
    b.step(20)
    a1, b1, u1 = a.get_fields()
    a2, b2, u2 = b.get_fields()
    assert np.allclose(flip(a1[0]), a2[0], atol=1e-12) and np.allclose(flip(b1[0]), b2[0], atol=1e-12)
    assert np.allclose(flip_u(u1[0]), u2[0], atol=1e-12)


@pytest.mark.parametrize("old,new", [
    ("    int keep = solid[0] ? 1 : 0; /* the open face: the particle moved along its axis */",
     "    int keep = solid[0] ? 0 : 1;"),
    ("    c[ax[flip]] = -c[ax[flip]];", "    c[ax[keep]] = -c[ax[keep]];"),
])
def test_slip_pins_catch_wrong_reflection(oracle_mod, old, new):
    """A reflection about the wrong plane, or from the wrong cell, planted in
    the oracle, breaks mass conservation or the frictionless stream."""
    with oracle_mod.planted(old, new):
        drift = _mass_drift(oracle_mod, 1.0)
        dev, _, _ = _channel_stream(oracle_mod, 1.0)
    assert drift > 1e-6 or dev > 1e-8, (drift, dev)
