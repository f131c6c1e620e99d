"""Permeability of a 1 % mixture in a packed-sphere array (Sec. 3.5).

The paper's porous medium is a fully packed array of spheres: a periodic cube of
side L holding one sphere of diameter L (the spheres of neighbouring cells
touch).  The pore space holds a mixture of 99 % component 1 and 1 % component
2 with equal viscosities, driven by a body force g along x.  The permeability
is nu U_D / g, with the Darcy velocity U_D = phi U (porosity phi, U the mean
velocity over the pore space).

With the original wetting model (wall model 1 here: a SOLID neighbour carries
rho^s alone) a wall that attracts the minority pushes the majority away from
it; the mixture thins next to the wall and slips, and the permeability grows
with the wetting strength.  Sec. 3.5 credits the modified model with removing
that, since the forces along walls are balanced between the components.  Wall
model 3 (the wall potential's force balanced between the components in every
cell) is that reading; wall model 2 (the neighbour carries the cell's own
density plus rho^s) is neutral at rho^s = 0 but still pushes the mixture off a
wetting wall.  Permeabilities are compared with the single-component value
k0(nu) of the same lattice, which itself depends on nu (the halfway
bounce-back wall sits at a viscosity-dependent position).

The force is set as g = c nu (the paper's "g nu = 0.024" is read as a
proportionality between g and nu, which keeps the Darcy velocity, and so the
Mach and Reynolds numbers, the same at every viscosity; a product held fixed
would drive the low-viscosity runs far beyond the lattice's speed range).
"""
from __future__ import annotations

import numpy as np

from . import workloads as W

T0 = 1.0 / 3.0


def sphere_array(L: int = 20):
    """One sphere of diameter L centred in a periodic cube of side L.
    Returns the cell types [L, L, L]."""
    c = np.arange(L) + 0.5 - L / 2.0
    r2 = c[None, None, :] ** 2 + c[None, :, None] ** 2 + c[:, None, None] ** 2
    return np.where(r2 < (L / 2.0) ** 2, W.SOLID, W.FLUID).astype(np.uint8)


def permeabilities(cases, L: int = 20, G: float = -2.2, wall_model: int = 2, c_force: float = 4e-4,
                   minority: float = 0.01, steps: int = 60000, tol: float = 1e-6, precision: str = "fp32",
                   check_every: int = 500):
    """cases: (nu, rho_s) pairs, all run as instances of one context (both
    components at viscosity nu) to steady state.  Returns, per case, the
    permeability nu U_D / g and the final residual; minority 0 gives the
    single-component value."""
    from . import lbm
    t = sphere_array(L)
    fluid = t != W.SOLID
    phi = float(fluid.mean())
    B = len(cases)
    r1 = np.where(fluid, 1.0 - minority, 0.0)
    r2 = np.where(fluid, minority, 0.0)
    u = np.zeros(t.shape + (3,))
    params = [dict(tau=(nu / T0 + 0.5, nu / T0 + 0.5), G=G, rho_s=rs, g=(c_force * nu, 0.0, 0.0))
              for nu, rs in cases]
    sim = lbm.Sim(L, L, L, params, precision=precision, wall_model=wall_model)
    sim.set_geometry(np.repeat(t[None], B, axis=0))
    sim.set_fields(np.repeat(r1[None], B, axis=0), np.repeat(r2[None], B, axis=0), np.repeat(u[None], B, axis=0))
    done, res = lbm.lbm_run_to_steady(sim.ctx, check_every, tol, steps, B)
    _, _, v = sim.get_fields()
    sim.close()
    out = []
    for k, (nu, rs) in enumerate(cases):
        U = float(v[k][..., 0][fluid].mean())
        g = c_force * nu
        out.append(dict(nu=nu, rho_s=rs, k=nu * phi * U / g, residual=float(res[k]), updates=int(done)))
    return out
