"""Closed forms the oracle is pinned to (no lattice Boltzmann arithmetic here).

* equation of state of the two-component pseudo-potential mixture, from the
  continuum limit of the interaction force (Eq. 7) with the force-stencil
  second moment sum_i ws_i c_i c_i = 2 T0 I:  p = T0 rho - 2 T0 G rho1 rho2;
* Laplace law: p_in - p_out = sigma / R (cylinder), 2 sigma / R (sphere);
* steady layered Poiseuille flow with a density-weighted mixture viscosity
  (Sec. 3.2): d/ds(rho nu du/ds) = -rho g, u = 0 at both walls.
"""
import numpy as np

T0 = 1.0 / 3.0
STENCIL_M2 = 2.0 * T0


def eos(rho1, rho2, G):
    return T0 * (rho1 + rho2) - STENCIL_M2 * G * rho1 * rho2


def layered_poiseuille(rho, nu, g):
    """Steady profile for piecewise-constant rho[j], nu[j] on cells j = 0..H-1
    (cell j spans s in [j, j+1], walls at s = 0 and s = H, no slip).

    Shear stress tau(s) = tau0 - g int_0^s rho, velocity u(s) = int_0^s
    tau / (rho nu); tau0 follows from u(H) = 0.  Returns u at the cell centres.
    """
    rho = np.asarray(rho, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    H = rho.size
    # u(s) = tau0 * A(s) - g * B(s), accumulated cell by cell
    A_edge = np.zeros(H + 1)
    B_edge = np.zeros(H + 1)
    Rm = np.concatenate([[0.0], np.cumsum(rho)])  # int_0^j rho
    A_c = np.zeros(H)
    B_c = np.zeros(H)
    for j in range(H):
        mu = rho[j] * nu[j]
        for frac, (Aout, Bout) in ((0.5, (A_c, B_c)), (1.0, (A_edge, B_edge))):
            d = frac
            a = A_edge[j] + d / mu
            b = B_edge[j] + (Rm[j] * d + rho[j] * d * d / 2.0) / mu
            if frac == 0.5:
                A_c[j], B_c[j] = a, b
            else:
                A_edge[j + 1], B_edge[j + 1] = a, b
    tau0 = g * B_edge[H] / A_edge[H]
    return tau0 * A_c - g * B_c


def single_phase_poiseuille(H, nu, g):
    s = np.arange(H) + 0.5
    return g * s * (H - s) / (2.0 * nu)


def golden(name):
    """Rows of a paper-value fixture under tests/golden/ (comment lines start
    with '#'; first remaining line is the header) as a list of dicts, numbers
    converted to float."""
    import csv
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    lines = [ln for ln in open(path) if ln.strip() and not ln.lstrip().startswith("#")]
    rows = []
    for r in csv.DictReader(lines):
        out = {}
        for k, v in r.items():
            try:
                out[k] = float(v)
            except ValueError:
                out[k] = v
        rows.append(out)
    return rows
