"""The seeded synthetic inputs keep the recipes they are quoted with: porosity
and minority fraction of the packed spheres, droplet volumes, wall rows and
boundary planes, and bit-for-bit reproducibility from the seed."""
import math

import numpy as np
import pytest

from paper_1711_03254_gb300 import workloads as W


def _fields_consistent(t, r1, r2, u):
    solid = t == W.SOLID
    assert np.all(r1[solid] == 0) and np.all(r2[solid] == 0) and np.all(u[solid] == 0)
    assert np.all((r1 + r2)[~solid] == 1.0)


def test_packed_spheres_recipe():
    t, r1, r2, u = W.packed_spheres(n=64, r=12.0, porosity=0.40, seed=3, droplet_r=4.0, minority=0.01)
    fluid = t != W.SOLID
    assert 0.39 <= fluid.mean() <= 0.40  # spheres are added until the porosity reaches 0.40
    frac2 = r2[fluid].sum() / fluid.sum()
    assert 0.01 <= frac2 < 0.03  # droplets are added until they fill 1 % of the pores
    assert set(np.unique(t)) <= {W.FLUID, W.SOLID}
    _fields_consistent(t, r1, r2, u)
    again = W.packed_spheres(n=64, r=12.0, porosity=0.40, seed=3, droplet_r=4.0, minority=0.01)
    assert all(np.array_equal(a, b) for a, b in zip((t, r1, r2, u), again))
    other = W.packed_spheres(n=64, r=12.0, porosity=0.40, seed=4, droplet_r=4.0, minority=0.01)
    assert not np.array_equal(t, other[0])


@pytest.mark.parametrize("nz", [1, 48])
def test_droplet_volume(nz):
    n, R = 48, 10.0
    t, r1, r2, u = W.droplet(n, n, nz, R)
    inside = r2 == 1.0
    ref = math.pi * R * R if nz == 1 else 4.0 / 3.0 * math.pi * R ** 3
    assert abs(inside.sum() - ref) / ref < 0.03
    assert np.all(t == W.FLUID)
    _fields_consistent(t, r1, r2, u)
    # centred: symmetric under reversing each axis
    for ax in range(3):
        assert np.array_equal(inside, np.flip(inside, axis=ax))


@pytest.mark.parametrize("layout", ["121", "12"])
def test_layered_channel_walls_and_layers(layout):
    nx, ny, nz = 4, 34, 3
    t, r1, r2, u = W.layered_channel(nx, ny, nz, layout=layout, wall_comp_nu=1.0, core_comp_nu=0.1, g=1e-6)
    assert np.all(t[:, 0, :] == W.SOLID) and np.all(t[:, ny - 1, :] == W.SOLID)
    assert np.all(t[:, 1:ny - 1, :] == W.FLUID)
    _fields_consistent(t, r1, r2, u)
    comp2_rows = np.flatnonzero(r2[0, :, 0] == 1.0)
    H = ny - 2
    if layout == "121":
        assert comp2_rows.size == H // 2 and r1[0, 1, 0] == 1.0 and r1[0, ny - 2, 0] == 1.0
    else:
        assert comp2_rows.size == H // 2 and r1[0, 1, 0] == 1.0 and r2[0, ny - 2, 0] == 1.0
    assert np.all(u[..., 1:] == 0) and np.all(u[:, 1:ny - 1, :, 0] > 0)


def test_rough_channel_planes():
    nx, ny, nz = 40, 20, 16
    t, r1, r2, u = W.rough_channel(nx, ny, nz, seed=4, invaded_length=8)
    assert np.all(t[:, 0, :] == W.SOLID) and np.all(t[0, :, :] == W.SOLID)
    assert set(np.unique(t[:, :, 0])) <= {W.INLET, W.SOLID} and np.any(t[:, :, 0] == W.INLET)
    assert set(np.unique(t[:, :, nx - 1])) <= {W.OUTLET, W.SOLID} and np.any(t[:, :, nx - 1] == W.OUTLET)
    assert np.all(r2[:, :, 8:] == 0) and np.all(r2[:, :, :8][t[:, :, :8] != W.SOLID] == 1.0)
    _fields_consistent(t, r1, r2, u)


@pytest.mark.parametrize("deg", [0.0, 30.0])
def test_inclined_droplet_rests_on_the_wall(deg):
    n, R = 48, 6.0
    t, r1, r2, u = W.inclined_droplet(n, deg, R)
    solid = t == W.SOLID
    drop = r2 == 1.0
    assert drop.sum() > 0.3 * 4.0 / 3.0 * math.pi * R ** 3
    # some droplet cell touches the wall (a SOLID face neighbour)
    touch = np.zeros_like(drop)
    for ax in range(3):
        for s in (1, -1):
            touch |= np.roll(solid, s, axis=ax)
    assert np.any(drop & touch)
    _fields_consistent(t, r1, r2, u)
