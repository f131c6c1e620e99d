"""Seeded synthetic inputs (geometry masks and initial fields).

This module holds no arithmetic of the lattice Boltzmann method: it only
builds cell-type masks and initial density / velocity fields.  Both the CUDA
path and the CPU oracle are fed from it.  Every random draw uses NumPy's
PCG64 generator with a fixed seed.

Cell types: 0 FLUID, 1 SOLID, 2 INLET, 3 OUTLET.  Arrays are shaped
[nz, ny, nx] (x fastest); velocities carry a trailing axis of 3.

Workloads (the paper's validation geometries, Sec. 3, in synthetic form):
  * ``droplet``        static droplet of component 2 in component 1 (Sec. 3.1);
  * ``layered_channel`` multi-component Poiseuille channel (Sec. 3.2);
  * ``packed_spheres`` porous medium of overlapping spheres with a 1 % minority
                       of droplets (stand-in for the packed-sphere geometry of
                       Sec. 3.5);
  * ``rough_channel``  channel with seeded wall bumps, with inlet and outlet
                       planes or periodic ends (the displacement / fingering
                       geometry family, Sec. 3.6-3.7);
  * ``inclined_droplet`` droplet on an inclined wall (Sec. 3.4).
"""
from __future__ import annotations

import math

import numpy as np

FLUID, SOLID, INLET, OUTLET = 0, 1, 2, 3


def _centres(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.float64) + 0.5


def droplet(nx: int, ny: int, nz: int, R: float, center=None, rho_major: float = 1.0,
            rho_minor: float = 0.0):
    """Sphere (nz > 1) or cylinder along z (nz == 1) of component 2 inside component 1.

    Cell centres sit at integer + 1/2; the default centre is the box centre.
    Returns (cell_type, rho1, rho2, u).
    """
    if center is None:
        center = (nx / 2.0, ny / 2.0, nz / 2.0)
    X = _centres(nx)[None, None, :] - center[0]
    Y = _centres(ny)[None, :, None] - center[1]
    Z = _centres(nz)[:, None, None] - center[2]
    r2 = X * X + Y * Y + (Z * Z if nz > 1 else 0.0 * Z)
    inside = np.broadcast_to(r2 < R * R, (nz, ny, nx))
    rho2 = np.where(inside, rho_major, rho_minor).astype(np.float64)
    rho1 = np.where(inside, rho_minor, rho_major).astype(np.float64)
    t = np.zeros((nz, ny, nx), dtype=np.uint8)
    u = np.zeros((nz, ny, nx, 3))
    return t, rho1, rho2, u


def layered_channel(nx: int, ny: int, nz: int, layout: str = "121", wall_comp_nu: float = 1.0,
                    core_comp_nu: float = 1.0, g: float = 0.0, rho_major: float = 1.0,
                    rho_minor: float = 0.0, analytic_velocity: bool = True):
    """Channel with SOLID rows y = 0 and y = ny-1 (walls at y = 0.5, ny - 1.5).

    layout "121": component 1 along both walls, component 2 in the middle half
    (interfaces at 1/4 and 3/4 of the gap); layout "12": component 1 in the lower
    half, component 2 in the upper half.  With ``analytic_velocity`` the initial
    u_x is the sharp-interface steady profile for body force g along x and the
    two kinematic viscosities (wall_comp_nu for component 1, core_comp_nu for
    component 2), so that slow viscous transients are skipped.
    Returns (cell_type, rho1, rho2, u).
    """
    t = np.zeros((nz, ny, nx), dtype=np.uint8)
    t[:, 0, :] = SOLID
    t[:, ny - 1, :] = SOLID
    H = ny - 2.0
    y = _centres(ny) - 1.0  # distance from the lower wall at y = 0.5 ... centre of row 1 is 0.5
    s = y  # position across the gap, 0 at the lower wall, H at the upper wall
    if layout == "121":
        comp2 = (s > H / 4.0) & (s < 3.0 * H / 4.0)
    elif layout == "12":
        comp2 = s > H / 2.0
    else:
        raise ValueError(layout)
    rho2_1d = np.where(comp2, rho_major, rho_minor)
    rho1_1d = np.where(comp2, rho_minor, rho_major)
    ux = np.zeros(ny)
    if analytic_velocity and g != 0.0:
        n1, n2 = wall_comp_nu, core_comp_nu
        if layout == "121":
            h = H / 2.0
            a = H / 4.0
            sc = s - h
            outer = g * (h * h - sc * sc) / (2.0 * n1)
            inner = g * (h * h - a * a) / (2.0 * n1) + g * (a * a - sc * sc) / (2.0 * n2)
            ux = np.where(np.abs(sc) <= a, inner, outer)
        else:
            d = H / 2.0
            # shear stress tau0 at the lower wall; continuity of u and stress at s = d
            tau0 = g * d * (1.0 / n1 + 3.0 / n2) / (2.0 * (1.0 / n1 + 1.0 / n2))
            lower = (tau0 * s - 0.5 * g * s * s) / n1
            ud = (tau0 * d - 0.5 * g * d * d) / n1
            upper = ud + (tau0 * (s - d) - 0.5 * g * (s * s - d * d)) / n2
            ux = np.where(s <= d, lower, upper)
        ux = np.where((s > 0) & (s < H), ux, 0.0)
    rho1 = np.broadcast_to(rho1_1d[None, :, None], (nz, ny, nx)).astype(np.float64).copy()
    rho2 = np.broadcast_to(rho2_1d[None, :, None], (nz, ny, nx)).astype(np.float64).copy()
    u = np.zeros((nz, ny, nx, 3))
    u[..., 0] = ux[None, :, None]
    rho1[t == SOLID] = 0.0
    rho2[t == SOLID] = 0.0
    u[t == SOLID] = 0.0
    return t, rho1, rho2, u


def _stamp_spheres(mask: np.ndarray, centres: np.ndarray, r: float, value=True) -> None:
    """Set mask to value inside periodic spheres of radius r (cell centres at +1/2)."""
    nz, ny, nx = mask.shape
    ri = int(math.ceil(r))
    off = np.arange(-ri - 1, ri + 2)
    for cz, cy, cx in centres:
        ix = np.floor(cx).astype(int) + off
        iy = np.floor(cy).astype(int) + off
        iz = np.floor(cz).astype(int) + off
        dx = (ix + 0.5 - cx)[None, None, :]
        dy = (iy + 0.5 - cy)[None, :, None]
        dz = (iz + 0.5 - cz)[:, None, None]
        inside = dx * dx + dy * dy + dz * dz < r * r
        sub = np.ix_(iz % nz, iy % ny, ix % nx)
        block = mask[sub]
        block[inside] = value
        mask[sub] = block


def packed_spheres(n: int = 256, r: float = 12.0, porosity: float = 0.40, seed: int = 3,
                   droplet_r: float = 4.0, minority: float = 0.01, ny: int | None = None,
                   nz: int | None = None):
    """Porous medium: overlapping spheres of radius r with uniform seeded centres
    added until the porosity reaches ``porosity`` (Boolean model; random
    sequential addition of non-overlapping spheres jams below porosity 0.6),
    then component-2 droplets of radius ``droplet_r`` at seeded fluid positions
    until they fill ``minority`` of the pore volume.  Periodic in all axes.
    Returns (cell_type, rho1, rho2, u).
    """
    nx = n
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    rng = np.random.default_rng(seed)
    solid = np.zeros((nz, ny, nx), dtype=bool)
    total = solid.size
    vol = 4.0 / 3.0 * math.pi * r ** 3
    while True:
        phi = 1.0 - solid.sum() / total
        if phi <= porosity:
            break
        # add a batch sized to close a good part of the remaining gap
        need = max(1, int(0.5 * (-math.log(porosity / phi)) * total / vol))
        c = rng.random((need, 3)) * np.array([nz, ny, nx])
        for k in range(need):
            _stamp_spheres(solid, c[k:k + 1], r)
            if 1.0 - solid.sum() / total <= porosity:
                break
    t = np.where(solid, SOLID, FLUID).astype(np.uint8)
    fluid_cells = np.flatnonzero(~solid.reshape(-1))
    drops = np.zeros_like(solid)
    target = minority * fluid_cells.size
    while (drops & ~solid).sum() < target:
        k = fluid_cells[rng.integers(fluid_cells.size)]
        z, rem = divmod(int(k), ny * nx)
        y, x = divmod(rem, nx)
        _stamp_spheres(drops, np.array([[z + 0.5, y + 0.5, x + 0.5]]), droplet_r)
    comp2 = drops & ~solid
    rho2 = np.where(comp2, 1.0, 0.0)
    rho1 = np.where(~solid & ~comp2, 1.0, 0.0)
    u = np.zeros((nz, ny, nx, 3))
    return t, rho1, rho2, u


def rough_channel(nx: int = 512, ny: int = 256, nz: int = 256, seed: int = 4, hmax: float = 4.0,
                  bumps_per_kcell: float = 0.5, invaded_length: int = 8, ends: str = "inlet_outlet"):
    """Channel along x with SOLID walls on the y and z faces and seeded
    hemispherical bumps of height <= hmax on those walls.  ends="inlet_outlet":
    an INLET plane at x = 0 and an OUTLET plane at x = nx - 1; ends="periodic":
    none (the channel is periodic along x and driven by a body force, as the
    displacement and fingering channels of Sec. 3.6 and 3.7 are).  The invading
    component 2 fills the first ``invaded_length`` planes; component 1
    (defending) fills the rest.  Returns (cell_type, rho1, rho2, u).
    """
    if ends not in ("inlet_outlet", "periodic"):
        raise ValueError("ends must be 'inlet_outlet' or 'periodic'")
    rng = np.random.default_rng(seed)
    solid = np.zeros((nz, ny, nx), dtype=bool)
    solid[:, 0, :] = True
    solid[:, ny - 1, :] = True
    solid[0, :, :] = True
    solid[nz - 1, :, :] = True
    wall_area = 2 * nx * (ny + nz)
    nb = int(bumps_per_kcell * wall_area / 1000.0)
    for _ in range(nb):
        h = rng.uniform(1.0, hmax)
        x = rng.uniform(0, nx)
        face = rng.integers(4)
        if face < 2:  # y walls
            z = rng.uniform(1, nz - 1)
            y = 1.0 if face == 0 else ny - 1.0
            c = np.array([[z, y, x]])
        else:
            y = rng.uniform(1, ny - 1)
            z = 1.0 if face == 2 else nz - 1.0
            c = np.array([[z, y, x]])
        _stamp_spheres(solid, c, h)
    t = np.where(solid, SOLID, FLUID).astype(np.uint8)
    if ends == "inlet_outlet":
        t[:, :, 0][~solid[:, :, 0]] = INLET
        t[:, :, nx - 1][~solid[:, :, nx - 1]] = OUTLET
    fluid = ~solid
    xs = np.arange(nx)[None, None, :]
    comp2 = fluid & (xs < invaded_length)
    rho2 = np.where(comp2, 1.0, 0.0)
    rho1 = np.where(fluid & ~comp2, 1.0, 0.0)
    u = np.zeros((nz, ny, nx, 3))
    return t, rho1, rho2, u


def inclined_droplet(n: int, incline_deg: float, R: float, thickness: float = 4.0):
    """Droplet of component 2 resting on a flat wall inclined by ``incline_deg``
    about the z axis (the inclined-channel geometry family of Sec. 3.4).
    The wall is the half-space below a plane through the lower quarter of the box.
    Returns (cell_type, rho1, rho2, u).
    """
    th = math.radians(incline_deg)
    nrm = np.array([-math.sin(th), math.cos(th), 0.0])  # wall normal (x, y, z)
    p0 = np.array([n / 2.0, n / 4.0, n / 2.0])
    X = _centres(n)[None, None, :]
    Y = _centres(n)[None, :, None]
    Z = _centres(n)[:, None, None]
    dist = (X - p0[0]) * nrm[0] + (Y - p0[1]) * nrm[1] + (Z - p0[2]) * nrm[2]
    solid = np.broadcast_to((dist < 0) & (dist > -n), (n, n, n)).copy()
    # keep the domain closed at the top too (channel)
    solid |= np.broadcast_to(dist > n / 2.0 + thickness, (n, n, n))
    c = p0 + nrm * (R * 0.6)
    r2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2
    comp2 = (r2 < R * R) & ~solid
    t = np.where(solid, SOLID, FLUID).astype(np.uint8)
    rho2 = np.where(comp2, 1.0, 0.0)
    rho1 = np.where(~solid & ~comp2, 1.0, 0.0)
    u = np.zeros((n, n, n, 3))
    return t, rho1, rho2, u
