"""Critical pressure of slug displacement (Sec. 3.6) on the GPU: a wetting slug
in the narrow section (height D) of a periodic channel of height 40 leaves it
once the body force exceeds the capillary pressure difference
2 sigma cos(theta) (1/D - 1/H) / (rho_0 L); the paper finds the simulated
critical acceleration within 10 % of that at D = 5 and 10, theta = 20 ... 80
degrees and the viscosity pairs (0.0017, 0.33), (0.33, 0.0017).  sigma is the
model's own (Laplace fit of 2-D droplets) and the wall potentials come from
the contact-angle calibration."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_03254_gb300 import build
    build.build()
    from paper_1711_03254_gb300 import displacement as DP, wetting as WT
    sigma, intercept = DP.surface_tension(-2.2)
    pairs = [(0.0017, 0.33), (0.33, 0.0017)]
    cal, _ = WT.Calibration.measure(pairs, list(np.round(np.linspace(-0.9, 0.9, 19), 3)), steps=30000, tol=1e-6,
                                    check_every=500)
    return DP, sigma, cal, pairs


def test_surface_tension_fit(setup):
    """The Laplace fit behind g_crit: sigma within 15 % of the paper's 0.11 at
    G = -2.2 (Sec. 3.1) and a small intercept."""
    DP, sigma, cal, pairs = setup
    assert abs(sigma - 0.11) / 0.11 < 0.15, sigma


def test_critical_acceleration_within_ten_percent(setup):
    DP, sigma, cal, pairs = setup
    cases = []
    for (n1, n2) in pairs:
        rs, th = cal.table[(n1, n2)]
        for D in (5, 10):
            for theta in (20, 40, 60, 80):
                if not (th.min() + 1.0 <= theta <= th.max() - 1.0):
                    continue
                cases.append(dict(nu1=n1, nu2=n2, D=D, theta=theta, rho_s=cal.rho_s(n1, n2, theta),
                                  g_ref=DP.g_crit_analytic(sigma, theta, D, 40, 160)))
    assert len(cases) >= 12
    first, remain = DP.critical_factors(cases)
    bad = [(c, f, r) for c, f, r in zip(cases, first, remain) if f is None or not (0.9 < f <= 1.1)]
    assert not bad, bad
