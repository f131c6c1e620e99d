"""Critical pressure for displacing a slug from a channel (Sec. 3.6).

A 2-D periodic channel of height H has a middle section of length Z narrowed
to height D.  A slug of component 2, which wets the walls (contact angle
theta < 90 degrees), fills the narrow section and reaches into the wide part
after it, one meniscus in each channel.  Capillarity pulls it into the narrow
section (its upstream meniscus then rests on the section's entrance); a body
force rho_0 g along the channel pushes it out.  It leaves once the pressure
drop the force builds over one period, rho_0 g L, exceeds the capillary
pressure difference of a meniscus of width D and one of width H (Eq. for the
critical pressure):

    P_crit = 2 sigma cos(theta) (1/D - 1/H),   g_crit = P_crit / (rho_0 L).

As in the paper the force is raised in stages, a fraction of the analytic
g_crit each (70 % ... 130 %), and the stage at which the slug leaves the narrow
section brackets the simulated critical acceleration.  The surface tension
sigma is this model's own, from the Laplace law (Delta p against 1/R of 2-D
droplets, Sec. 3.1), and the wall potential of each wanted angle comes from the
contact-angle calibration of Sec. 3.3 (wetting.Calibration).
"""
from __future__ import annotations

import math

import numpy as np

from . import workloads as W

T0 = 1.0 / 3.0
STAGES = (0.7, 0.9, 0.95, 1.0, 1.05, 1.1, 1.3)


def constricted_channel(L: int = 160, H: int = 40, D: int = 10, Z: int = 52, slug: int = 16):
    """SOLID rows y = 0 and H + 1; x in [x0, x0 + Z) narrowed to the rows
    [y_lo, y_lo + D) (centred).  Component 2 fills the whole narrow section and
    the first `slug` columns of the wide channel after it, so that one meniscus
    sits in each channel (the configuration of the critical pressure; a slug
    inside the narrow section alone would have to push its meniscus past the
    step's corner, a higher barrier); component 1 elsewhere.  Returns
    (cell_type, rho1, rho2, u) shaped [1, H + 2, L] and the narrow-section mask
    [H + 2, L]."""
    ny = H + 2
    x0 = (L - Z) // 2
    y_lo = 1 + (H - D) // 2
    t = np.zeros((1, ny, L), dtype=np.uint8)
    t[:, 0, :] = W.SOLID
    t[:, ny - 1, :] = W.SOLID
    xs = np.arange(L)[None, :]
    ys = np.arange(ny)[:, None]
    in_narrow_x = (xs >= x0) & (xs < x0 + Z)
    open_rows = (ys >= y_lo) & (ys < y_lo + D)
    t[0][in_narrow_x & ~open_rows] = W.SOLID
    narrow = in_narrow_x & open_rows
    fluid = t[0] != W.SOLID
    slug_cells = narrow | (fluid & (xs >= x0 + Z) & (xs < x0 + Z + slug))
    rho2 = np.where(slug_cells, 1.0, 0.0)[None]
    rho1 = np.where(fluid & ~slug_cells, 1.0, 0.0)[None]
    u = np.zeros(t.shape + (3,))
    return t, rho1, rho2, u, narrow


def g_crit_analytic(sigma: float, theta_deg: float, D: float, H: float, L: float, rho0: float = 1.0) -> float:
    """Critical acceleration of the capillary pressure difference (Sec. 3.6)."""
    return 2.0 * sigma * math.cos(math.radians(theta_deg)) * (1.0 / D - 1.0 / H) / (rho0 * L)


def surface_tension(G: float = -2.2, radii=(10, 16, 24), steps: int = 8000, precision: str = "fp32"):
    """sigma of this model at coupling G: slope of Delta p against 1/R of
    cylindrical droplets in periodic boxes 5R (pressure from the equation of
    state p = T0 rho - 2 T0 G rho_1 rho_2 at the centre and at a corner)."""
    from . import lbm
    dps = []
    for R in radii:
        n = int(5 * R)
        t, r1, r2, u = W.droplet(n, n, 1, R)
        sim = lbm.Sim(n, n, 1, [dict(tau=(1.0, 1.0), G=G)], precision=precision)
        sim.set_geometry(t[None])
        sim.set_fields(r1[None], r2[None], u[None])
        sim.step(steps)
        a, b, _ = sim.get_fields()
        sim.close()
        p = T0 * (a[0, 0] + b[0, 0]) - 2.0 * T0 * G * a[0, 0] * b[0, 0]
        c = n // 2
        dps.append(p[c - 1:c + 1, c - 1:c + 1].mean() - p[0, 0])
    sigma, intercept = np.polyfit(1.0 / np.asarray(radii, float), np.asarray(dps), 1)
    return float(sigma), float(intercept)


def critical_factors(cases, G: float = -2.2, L: int = 160, H: int = 40, Z: int = 52, slug: int = 16,
                     stages=STAGES, steps_per_stage: int = 80000, settle: float = 0.5, precision: str = "fp32",
                     drain: float = 0.05, leave: float = 0.5):
    """cases: dicts with nu1, nu2, rho_s, D, g_ref.  All cases run as instances
    of one context.  A settling stage at `settle` * g_ref (half a stage) lets
    each slug find its pinned position; then stage k applies
    g = stages[k] * g_ref along x for steps_per_stage updates.  A case counts
    as displaced at the first stage over which the slug's component 2 in the
    narrow section falls by more than `drain` (of its initial amount), or to
    below `leave` of it (a slug held by capillarity stays put at a force below
    the critical one; the fields turning non-finite counts as displaced: the
    carrier then accelerates without bound).  Returns, per case, the first
    displacing stage factor (None if never) and the remaining fraction after
    the settling stage and after every stage."""
    from . import lbm
    geos = [constricted_channel(L, H, c["D"], Z, slug) for c in cases]
    t = np.stack([g[0] for g in geos])
    r1 = np.stack([g[1] for g in geos])
    r2 = np.stack([g[2] for g in geos])
    u = np.stack([g[3] for g in geos])
    masks = [g[4] for g in geos]
    m0 = [float(r2[k, 0][masks[k]].sum()) for k in range(len(cases))]

    def params(f):
        return [dict(tau=(c["nu1"] / T0 + 0.5, c["nu2"] / T0 + 0.5), G=G, rho_s=c["rho_s"],
                     g=(f * c["g_ref"], 0.0, 0.0)) for c in cases]

    def remaining(sim):
        _, b, _ = sim.get_fields()
        out = []
        for k in range(len(cases)):
            bk = b[k, 0]
            out.append(float(bk[masks[k]].sum()) / m0[k] if np.isfinite(bk).all() else 0.0)
        return out

    sim = lbm.Sim(L, H + 2, 1, params(settle), precision=precision)
    sim.set_geometry(t)
    sim.set_fields(r1, r2, u)
    sim.step(steps_per_stage // 2)
    prev = remaining(sim)
    first = [None] * len(cases)
    remain = [[p] for p in prev]
    for f in stages:
        sim.set_params(params(f))
        sim.step(steps_per_stage)
        now = remaining(sim)
        for k in range(len(cases)):
            remain[k].append(now[k])
            if first[k] is None and (prev[k] - now[k] > drain or now[k] < leave):
                first[k] = f
        prev = now
    sim.close()
    return first, remain
