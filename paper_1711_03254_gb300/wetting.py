"""Contact-angle calibration theta = L(nu_1, nu_2, rho^s) and its inverse (Sec. 3.3).

The paper relates the contact angle to the single wall potential rho^s of
Eq. 11 with a static slug between flat plates: a 2-D channel of height 32 and
length 128, periodic along the walls, half of it filled with component 2.  It
formulates theta as a function of the two viscosities and rho^s from those
runs and inverts that function to find the rho^s of a wanted angle.

Here every (viscosity pair, rho^s) case is one instance of a batched context
(all of them advance in the same launches); at steady state each slug's two
menisci are measured by a circle fit of the interface phi = (rho_1 - rho_2) /
(rho_1 + rho_2) = 0 (interface positions per row by linear interpolation, the
rows next to the walls left out).  The contact angle is the angle between the
circle and the wall, measured through component 2:
    cos(theta) = +-(W / 2) / R,
W the wall distance, R the fitted radius, + when the circle's centre lies on
the component-1 side (component 2 wets the wall, theta < 90 degrees).

Also measured: the thin film, the density of component 2 in the fluid row next
to a wall, halfway along the component-1 region (the quantity Sec. 3.3 uses to
compare the original and the modified wetting model).
"""
from __future__ import annotations

import math

import numpy as np

from . import workloads as W

T0 = 1.0 / 3.0


def slug_channel(L: int = 128, H: int = 32):
    """SOLID rows y = 0 and H - 1 (walls at y = 1 and y = H - 1 in cell-face
    coordinates), component 2 in L/4 <= x < 3L/4, component 1 elsewhere.
    Returns (cell_type, rho1, rho2, u) shaped [1, H, L] (one plane)."""
    t = np.zeros((1, H, L), dtype=np.uint8)
    t[:, 0, :] = W.SOLID
    t[:, H - 1, :] = W.SOLID
    x = np.arange(L)[None, None, :]
    slug = (x >= L // 4) & (x < 3 * L // 4) & (t != W.SOLID)
    rho2 = np.where(slug, 1.0, 0.0)
    rho1 = np.where((t != W.SOLID) & ~slug, 1.0, 0.0)
    u = np.zeros(t.shape + (3,))
    return t, rho1, rho2, u


def _interface_x(phi_row: np.ndarray, lo: int, hi: int) -> float | None:
    """x (cell-centre coordinates, cell i at i + 1/2) where phi crosses zero in
    [lo, hi), by linear interpolation; None if it does not."""
    for i in range(lo, hi - 1):
        a, b = phi_row[i], phi_row[i + 1]
        if a == 0.0:
            return i + 0.5
        if (a < 0.0) != (b < 0.0):
            return i + 0.5 + a / (a - b)
    return None


def _fit_circle(xs: np.ndarray, ys: np.ndarray):
    """Algebraic least-squares circle (x - a)^2 + (y - b)^2 = R^2."""
    A = np.column_stack([xs, ys, np.ones_like(xs)])
    rhs = -(xs * xs + ys * ys)
    (D, E, F), *_ = np.linalg.lstsq(A, rhs, rcond=None)
    a, b = -D / 2.0, -E / 2.0
    R2 = a * a + b * b - F
    return a, b, math.sqrt(R2) if R2 > 0 else float("inf")


def contact_angles(rho1: np.ndarray, rho2: np.ndarray, t: np.ndarray, skip_rows: int = 2):
    """Contact angles (degrees, through component 2) of the two menisci of a
    slug in a channel [H, L] with SOLID rows 0 and H - 1.  Rows within
    `skip_rows` of a wall are left out of the fit."""
    H, L = t.shape
    rho = rho1 + rho2
    phi = np.where(rho > 0, (rho1 - rho2) / np.where(rho > 0, rho, 1.0), 0.0)
    Wd = H - 2.0  # distance between the walls at y = 1 and y = H - 1
    out = []
    # left meniscus: component 1 (phi > 0) at smaller x; right: at larger x
    for side, (lo, hi) in (("left", (0, L // 2)), ("right", (L // 2, L))):
        xs, ys = [], []
        for y in range(1 + skip_rows, H - 1 - skip_rows):
            xi = _interface_x(phi[y], lo, hi)
            if xi is not None:
                xs.append(xi)
                ys.append(y + 0.5)
        xs, ys = np.asarray(xs), np.asarray(ys)
        if xs.size < 3 or np.ptp(xs) < 1e-9:
            out.append(90.0)
            continue
        a, b, R = _fit_circle(xs, ys)
        c = min(1.0, (Wd / 2.0) / R)
        ang = math.degrees(math.acos(c))
        # centre on the component-1 side: right meniscus a > x_mean, left a < x_mean
        centre_in_1 = (a > xs.mean()) if side == "right" else (a < xs.mean())
        out.append(ang if centre_in_1 else 180.0 - ang)
    return out


def thin_film(rho2: np.ndarray, t: np.ndarray) -> float:
    """Density of component 2 in the fluid rows next to the walls, halfway
    along the component-1 region (x = 0, the middle of the periodic outside
    region of slug_channel), mean of both walls."""
    H, L = t.shape
    return 0.5 * (rho2[1, 0] + rho2[H - 2, 0])


def run_slugs(cases, steps: int = 20000, G: float = -2.2, L: int = 128, H: int = 32, precision: str = "fp32",
              wall_model: int = 2, check_every: int = 500, tol: float = 1e-7):
    """Static slugs for cases [(nu_1, nu_2, rho_s), ...], all instances of one
    batched context, run to steady state (residual tol) or `steps` updates.
    Returns a list of dicts: theta (mean of both menisci), theta_left/right,
    film, residual."""
    from . import lbm
    t, r1, r2, u = slug_channel(L, H)
    B = len(cases)
    params = [dict(tau=(nu1 / T0 + 0.5, nu2 / T0 + 0.5), G=G, rho_s=rs) for nu1, nu2, rs in cases]
    sim = lbm.Sim(L, H, 1, params, precision=precision, wall_model=wall_model)
    sim.set_geometry(np.repeat(t[None], B, axis=0))
    sim.set_fields(np.repeat(r1[None], B, axis=0), np.repeat(r2[None], B, axis=0), np.repeat(u[None], B, axis=0))
    done, res = lbm.lbm_run_to_steady(sim.ctx, check_every, tol, steps, B)
    a, b, _ = sim.get_fields()
    sim.close()
    out = []
    for k in range(B):
        th = contact_angles(a[k, 0], b[k, 0], t[0])
        out.append(dict(nu1=cases[k][0], nu2=cases[k][1], rho_s=cases[k][2], theta=float(np.mean(th)),
                        theta_left=th[0], theta_right=th[1], film=float(thin_film(b[k, 0], t[0])),
                        residual=float(res[k]), updates=int(done)))
    return out


class Calibration:
    """theta(rho^s) tables per viscosity pair and their inverse.  theta falls
    monotonically as rho^s grows (rho^s > 0 makes the wall act as component 2,
    which then wets it); the inverse interpolates linearly between the
    calibrated points."""

    def __init__(self, table: dict):
        # table[(nu1, nu2)] = (rho_s values ascending, theta values)
        self.table = {k: (np.asarray(v[0], float), np.asarray(v[1], float)) for k, v in table.items()}

    @classmethod
    def measure(cls, nu_pairs, rho_s_values, **kw):
        cases = [(n1, n2, rs) for (n1, n2) in nu_pairs for rs in rho_s_values]
        res = run_slugs(cases, **kw)
        table = {}
        for (n1, n2) in nu_pairs:
            rows = sorted([r for r in res if (r["nu1"], r["nu2"]) == (n1, n2)], key=lambda r: r["rho_s"])
            table[(n1, n2)] = ([r["rho_s"] for r in rows], [r["theta"] for r in rows])
        return cls(table), res

    def theta(self, nu1, nu2, rho_s) -> float:
        rs, th = self.table[(nu1, nu2)]
        return float(np.interp(rho_s, rs, th))

    def rho_s(self, nu1, nu2, theta) -> float:
        """Wall potential giving contact angle theta (degrees) for this pair."""
        rs, th = self.table[(nu1, nu2)]
        order = np.argsort(th)
        return float(np.interp(theta, th[order], rs[order]))
