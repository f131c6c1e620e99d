"""The learned warm start against the plain start, in the configuration of
the full experiment restricted to its 64^3 test (about three minutes):
64^3 droplets on inclined walls (320 training cases run to their steady
state by the solver, 2000 Adam iterations), then 6 held-out cases run to
the same residual from both starts.  The warm start must need
fewer updates in total and converge to the same state (largest density
difference between the two converged fields below 0.05).  The full-size
experiment (also 128^3 test cases, and a fluid-at-rest variant) is
paper_1711_03254_gb300.warmstart."""
import pytest

pytestmark = pytest.mark.gpu

VARIANT = "warm"


def test_warm_start_cuts_updates_to_steady():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_03254_gb300 import build
    build.build()
    from paper_1711_03254_gb300 import warmstart
    res = warmstart.experiment(n_train=320, n_test=6, S_train=64, test_sizes=(64,), gen_max_steps=25000, iters=2000,
                               tol=1e-5, max_steps=40000, log=lambda *a: None, variants=((VARIANT, True),))
    rows = res["tests"][0]["rows"]
    plain = sum(r["plain_steps"] for r in rows)
    warm = sum(r[f"{VARIANT}_steps"] for r in rows)
    print("updates to steady, plain / warm:", [(r["plain_steps"], r[f"{VARIANT}_steps"]) for r in rows], plain, warm)
    assert warm < plain, [(r["plain_steps"], r[f"{VARIANT}_steps"]) for r in rows]
    for r in rows:
        if r["plain_res"] <= 1e-5 and r[f"{VARIANT}_res"] <= 1e-5:
            assert r[f"{VARIANT}_max_density_diff"] < 0.05, r
