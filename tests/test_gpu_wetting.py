"""Contact-angle calibration of Sec. 3.3 on the GPU: static slugs in the 128 x 32
channel, theta = L(nu_1, nu_2, rho^s) measured per viscosity pair, inverted,
and checked by running slugs at the inverted wall potentials (the paper's
simulated-against-expected angle check); the thin film of the original and the
modified wetting model."""
import numpy as np
import pytest

from paper_1711_03254_gb300 import wetting as WT

pytestmark = pytest.mark.gpu

# viscosity pairs of Sec. 3.3's range (nu from 0.0017 to 0.33, ratio up to 194)
PAIRS = [(1 / 6, 1 / 6), (0.33, 0.033), (0.033, 0.33), (0.33, 0.0017), (0.0017, 0.33)]
GRID = list(np.round(np.linspace(-0.6, 0.6, 13), 3))


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_03254_gb300 import build
    build.build()
    from paper_1711_03254_gb300 import lbm as mod
    return mod


@pytest.fixture(scope="module")
def calibration(lbm):
    cal, res = WT.Calibration.measure(PAIRS, GRID, steps=30000, tol=1e-6, check_every=500)
    return cal, res


def test_calibration_is_monotone_and_neutral(calibration):
    """theta falls monotonically as rho^s grows for every pair, and rho^s = 0
    with equal viscosities is neutral (90 degrees)."""
    cal, _ = calibration
    for (n1, n2), (rs, th) in cal.table.items():
        assert np.all(np.diff(th) < 0), (n1, n2, th)
    assert abs(cal.theta(1 / 6, 1 / 6, 0.0) - 90.0) < 0.1


def test_inverse_reproduces_expected_angles(lbm, calibration):
    """Slugs run at the wall potential the inverse gives for 40 ... 140
    degrees (inside every pair's calibrated range) show that angle within 2
    degrees."""
    cal, _ = calibration
    expected = [40.0, 60.0, 90.0, 120.0, 140.0]
    cases = [(n1, n2, cal.rho_s(n1, n2, th)) for (n1, n2) in PAIRS for th in expected]
    out = WT.run_slugs(cases, steps=30000, tol=1e-6, check_every=500)
    for r, th in zip(out, expected * len(PAIRS)):
        assert abs(r["theta"] - th) < 2.0, (r, th)
        assert abs(r["theta_left"] - r["theta_right"]) < 0.5


def test_thin_film_original_against_modified(lbm):
    """At rho^s = 0.3 the component-2 film along the walls of the component-1
    region is at least five times thinner with the modified wall models (2,
    and 3 with its balanced wall forces) than with the original one (1), for
    equal and for very different viscosities (Sec. 3.3, thin film)."""
    cases = [(1 / 6, 1 / 6, 0.3), (0.33, 0.0017, 0.3)]
    f1 = WT.run_slugs(cases, steps=20000, tol=1e-6, wall_model=1)
    for wm in (2, 3):
        fm = WT.run_slugs(cases, steps=20000, tol=1e-6, wall_model=wm)
        for a, b in zip(f1, fm):
            assert b["film"] * 5.0 < a["film"], (wm, a, b)


def test_balanced_walls_narrow_the_angle_range(lbm):
    """Wall model 3 acts only where both components meet the wall, so its
    angles stay near 90 degrees: within 65 ... 115 degrees for |rho^s| <= 0.6
    at equal viscosities (measured 73.2 ... 106.8), where model 2 spans
    23.6 ... 156.4; and theta(rho^s) is still monotone."""
    grid = [-0.6, -0.3, 0.0, 0.3, 0.6]
    out = WT.run_slugs([(1 / 6, 1 / 6, rs) for rs in grid], steps=30000, tol=1e-6, wall_model=3)
    th = [r["theta"] for r in out]
    assert all(65.0 < v < 115.0 for v in th), th
    assert all(a > b for a, b in zip(th, th[1:])), th
    assert abs(th[2] - 90.0) < 0.5, th


def test_slug_matches_oracle(lbm, oracle_mod):
    """The FP64 slug equals the oracle's after 1500 updates, and so does its
    measured contact angle."""
    t, r1, r2, u = WT.slug_channel()
    p = [dict(tau=(0.7, 1.5), G=-2.2, rho_s=0.3)]
    sim = lbm.Sim(128, 32, 1, p, precision="fp64")
    sim.set_geometry(t[None])
    sim.set_fields(r1[None], r2[None], u[None])
    sim.step(1500)
    a, b, _ = sim.get_fields()
    ref = oracle_mod.OracleSim(128, 32, 1, p)
    ref.set_geometry(t[None])
    ref.set_fields(r1[None], r2[None], u[None])
    ref.step(1500)
    ra, rb, _ = ref.get_fields()
    assert np.abs(a - ra).max() < 1e-12 and np.abs(b - rb).max() < 1e-12
    th, tho = WT.contact_angles(a[0, 0], b[0, 0], t[0]), WT.contact_angles(ra[0, 0], rb[0, 0], t[0])
    assert np.allclose(th, tho, atol=1e-6)
