"""Learned warm start of the two-component solver (data generation with the
solver, training of the U-Net, and the steps-to-steady comparison).

Problem family: a droplet of component 2 on an inclined flat wall (the
inclined-channel geometry of Sec. 3.4), parameters drawn from a seeded
generator:
  * contact angle theta ~ U[30 deg, 150 deg], turned into the wall potential
    rho^s by the contact-angle calibration of Sec. 3.3 (static slugs at this
    family's coupling, wetting.Calibration; interpolated in log10 of the
    viscosity ratio between the calibrated pairs);
  * inclination ~ U[0 deg, 45 deg];
  * viscosity ratio ~ logU[1, 1000] with nu_high = 1.7 (nu_low >= 0.0017),
    the droplet taking the low or the high viscosity at random;
  * a body force of magnitude ~ U[0, 1e-4] along the wall's inward normal
    (pressing the fluid onto the wall, so the steady state stays static);
  * G = -1.8 (both components stay stable down to nu = 0.0017 at this
    coupling; at -2.2 the family diverges at the low viscosities).

The training target is the solver's state once every residual of its batch
is below the tolerance (or after a cap on the updates), run from the plain
initial state (sharp droplet, fluid at rest).  The warm start runs the
network at 64^3 (inputs sampled every second cell for 128^3 problems) and
upsamples its output by nearest neighbours; the solver then runs from those
fields to the same residual as from the plain state.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import lbm, surrogate, wetting, workloads as W

G_WS = -1.8
NU_HIGH = 1.7
G_NORMAL_MAX = 1e-4
# viscosity ratios of the calibration; each with the droplet (component 2)
# taking the low or the high viscosity
CAL_RATIOS = (1.0, 10.0, 100.0, 1000.0)
CAL_GRID = tuple(np.round(np.linspace(-0.6, 0.6, 13), 3))
_CAL = {}


def _pair(ratio: float, drop_low: bool):
    low = NU_HIGH / ratio
    return (NU_HIGH, low) if drop_low else (low, NU_HIGH)


def family_calibration(steps: int = 30000):
    """theta(rho^s) of the family's viscosity pairs at its coupling (cached)."""
    if "cal" not in _CAL:
        pairs = [_pair(r, dl) for r in CAL_RATIOS for dl in (True, False)]
        pairs = list(dict.fromkeys(pairs))
        _CAL["cal"], _CAL["runs"] = wetting.Calibration.measure(pairs, list(CAL_GRID), steps=steps, tol=1e-6,
                                                                 check_every=500, G=G_WS)
    return _CAL["cal"]


def rho_s_for(theta: float, ratio: float, drop_low: bool) -> float:
    """Wall potential for contact angle theta at this viscosity ratio: the
    calibrated inverses at the neighbouring ratios, interpolated in log10."""
    cal = family_calibration()
    lr = math.log10(ratio)
    lg = [math.log10(r) for r in CAL_RATIOS]
    k = min(max(int(np.searchsorted(lg, lr)) - 1, 0), len(lg) - 2)
    w = (lr - lg[k]) / (lg[k + 1] - lg[k])
    a = cal.rho_s(*_pair(CAL_RATIOS[k], drop_low), theta)
    b = cal.rho_s(*_pair(CAL_RATIOS[k + 1], drop_low), theta)
    return (1.0 - w) * a + w * b


def sample_cases(n: int, seed: int, with_rho_s: bool = True):
    rng = np.random.default_rng(seed)
    cases = []
    for _ in range(n):
        ratio = 10 ** rng.uniform(0.0, 3.0)
        drop_low = bool(rng.random() < 0.5)
        theta = float(rng.uniform(30.0, 150.0))
        c = dict(theta=theta, incline=float(rng.uniform(0.0, 45.0)), nu=_pair(ratio, drop_low), ratio=float(ratio),
                 drop_low=drop_low, g_n=float(rng.uniform(0.0, G_NORMAL_MAX)))
        if with_rho_s:
            c["rho_s"] = rho_s_for(theta, ratio, drop_low)
        cases.append(c)
    return cases


def _normal(c):
    th = math.radians(c["incline"])
    return np.array([-math.sin(th), math.cos(th), 0.0])  # the wall's inward normal (x, y, z)


def case_params(c):
    g = -c["g_n"] * _normal(c)
    return dict(tau=(c["nu"][0] * 3 + 0.5, c["nu"][1] * 3 + 0.5), G=G_WS, rho_s=c["rho_s"], g=tuple(float(v) for v in g))


def case_geometry(c, S: int):
    return W.inclined_droplet(S, c["incline"], R=S / 8.0)


def case_inputs(c, S: int):
    t, r1, r2, u = case_geometry(c, S)
    return surrogate.encode_inputs(t, c["theta"], c["ratio"], c["incline"], c["g_n"], r2), t, r1, r2, u


def generate(cases, S: int = 64, max_steps: int = 40000, tol: float = 3e-6, batch: int = 32, precision: str = "fp32",
             check_every: int = 500):
    """Run the solver from the plain initial state of every case towards its
    steady state: each batch of instances advances in chunks of check_every
    updates until every instance has its residual <= tol or has diverged, or
    max_steps is reached.  Returns (inputs, targets, masks, kept case indices,
    residuals of the kept cases); cases whose state is not finite, or whose
    velocity reaches the sound speed, are left out."""
    X, Y, M, kept, resid = [], [], [], [], []
    for k0 in range(0, len(cases), batch):
        cs = cases[k0:k0 + batch]
        geo = [case_geometry(c, S) for c in cs]
        t = np.stack([g[0] for g in geo])
        sim = lbm.Sim(S, S, S, [case_params(c) for c in cs], precision=precision)
        sim.set_geometry(t)
        sim.set_fields(np.stack([g[1] for g in geo]), np.stack([g[2] for g in geo]), np.stack([g[3] for g in geo]))
        sim.reduce(allow_diverged=True)  # residual snapshot
        bad = np.zeros(len(cs), bool)
        res = np.full(len(cs), np.inf)
        done = 0
        while done < max_steps:
            sim.step(check_every)
            done += check_every
            red = sim.reduce(allow_diverged=True)
            res = red[:, 5]
            bad |= ~np.isfinite(red).all(axis=1) | (red[:, 6] >= 1 / math.sqrt(3))
            if np.all(bad | (res <= tol)):
                break
        r1, r2, u = sim.get_fields()
        sim.close()
        for j, c in enumerate(cs):
            if bad[j] or not all(np.isfinite(a[j]).all() for a in (r1, r2, u)):
                continue
            X.append(surrogate.encode_inputs(geo[j][0], c["theta"], c["ratio"], c["incline"], c["g_n"], geo[j][2]))
            Y.append(surrogate.encode_targets(r1[j], r2[j], u[j]))
            M.append((geo[j][0] != W.SOLID).astype(np.uint8))
            kept.append(k0 + j)
            resid.append(float(res[j]))
    return np.stack(X), np.stack(Y), np.stack(M), kept, resid


def train(net, X, Y, M, iters: int, lr: float = 1e-3, seed: int = 0, log_every: int = 50):
    """Adam on random mini-batches of net.N samples; returns the loss history."""
    import torch
    rng = np.random.default_rng(seed)
    dev = torch.device("cuda")
    Xd = torch.from_numpy(X).to(dev)
    Yd = torch.from_numpy(Y).to(dev)
    Md = torch.from_numpy(M).to(dev)
    wch = torch.tensor([1.0, 10.0, 1.0, 1.0, 1.0], dtype=torch.float32, device=dev)
    hist = []
    for it in range(iters):
        idx = torch.from_numpy(rng.choice(len(X), size=net.N, replace=False)).to(dev)
        x = Xd.index_select(0, idx).contiguous()
        y = Yd.index_select(0, idx).contiguous()
        m = Md.index_select(0, idx).contiguous()
        net.forward(x)
        loss = net.loss_and_grad(y, m, wch)
        net.backward()
        a = lr * 0.5 * (1 + math.cos(math.pi * it / max(1, iters)))
        net.adam_step(lr=a)
        if it % log_every == 0 or it == iters - 1:
            lv = float(loss.item())
            hist.append((it, lv))
            if not math.isfinite(lv):
                raise FloatingPointError(f"training loss is not finite at iteration {it}")
    return hist


def predict(net, x):
    """Network output for one input at the network's size (FP32 numpy [S,S,S,CIN])."""
    import torch
    xb = torch.zeros((net.N,) + x.shape, dtype=torch.float32, device="cuda")
    xb[0] = torch.from_numpy(x).cuda()
    out = net.forward(xb)
    return out[0].float().cpu().numpy()


def warm_fields(net, c, S: int, velocity: bool = True):
    """Initial fields for an S^3 case from the network: run at the network's
    size net.S (inputs sampled every S / net.S cells) and upsample the output
    by nearest neighbours.  S must be a multiple of net.S.  velocity=False
    keeps the predicted densities and starts the fluid at rest."""
    if S % net.S:
        raise ValueError("warm_fields: the case size must be a multiple of the network size")
    x, t, r1, r2, u = case_inputs(c, S)
    f = S // net.S
    if f == 1:
        out = predict(net, x)
    else:
        o = predict(net, np.ascontiguousarray(x[::f, ::f, ::f]))
        out = o.repeat(f, 0).repeat(f, 1).repeat(f, 2)
    r1p, r2p, up = surrogate.decode_fields(out, t)
    if not velocity:
        up = np.zeros_like(up)
    return t, (r1p, r2p, up)


def steps_to_steady(c, S, init, tol, check_every=100, max_steps=20000, precision="fp32"):
    """(updates, wall seconds, final residual, fields) to reach residual <= tol
    from `init`; a run that diverges (a non-finite value or |u_F| at the
    sound speed) returns the residual inf."""
    t, (r1, r2, u) = init
    sim = lbm.Sim(S, S, S, [case_params(c)], precision=precision)
    sim.set_geometry(t[None])
    sim.set_fields(r1[None], r2[None], u[None])
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        done, res = lbm.lbm_run_to_steady(sim.ctx, check_every, tol, max_steps, 1)
        res0 = float(res[0])
    except lbm.LbmError as e:
        if e.status != 4:
            raise
        done, res0 = max_steps, math.inf
    dt = time.perf_counter() - t0
    fields = sim.get_fields()
    sim.close()
    return done, dt, res0, fields


def experiment(n_train=2000, n_test=32, S_train=64, test_sizes=(64, 128), gen_max_steps=40000, iters=2000, batch=4,
               lr=1e-3, tol=3e-6, check_every=100, max_steps=60000, seed_train=5, seed_test=6, log=print,
               variants=(("warm", True), ("warm_rho", False)), n_test_large=8):
    """Generate, train, and compare updates / wall time to steady state from
    the plain and the learned initial fields (n_test cases at the training
    size, n_test_large at the larger test sizes).  Returns a summary dict."""
    import torch
    t0 = time.perf_counter()
    X, Y, M, kept, gres = generate(sample_cases(n_train, seed_train), S=S_train, max_steps=gen_max_steps, tol=tol)
    t_gen = time.perf_counter() - t0
    log(f"generated {len(X)} steady states at {S_train}^3 in {t_gen:.1f} s "
        f"({n_train - len(kept)} of {n_train} cases left out: not finite or |u| >= c_s; "
        f"median residual {np.median(gres):.2e})")
    net = surrogate.UNet3D(batch, S_train, seed=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = train(net, X, Y, M, iters, lr=lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    flops = 3.0 * net.flops_per_sample() * batch * iters
    log(f"trained {iters} iterations in {t_train:.1f} s ({flops / t_train / 1e12:.1f} TFLOP/s), "
        f"loss {hist[0][1]:.4g} -> {hist[-1][1]:.4g}")
    tests = []
    for S_test in test_sizes:
        rows = []
        want = n_test if S_test == S_train else min(n_test, n_test_large)
        skipped = 0
        for c in sample_cases(4 * want, seed_test):
            if len(rows) == want:
                break
            x, t, r1, r2, u = case_inputs(c, S_test)
            plain = steps_to_steady(c, S_test, (t, (r1, r2, u)), tol, check_every, max_steps)
            if not math.isfinite(plain[2]):
                # the family is sampled "where stable": a case the solver itself
                # cannot run is left out of the comparison (and counted)
                skipped += 1
                log(f"{S_test}^3 case skipped: the plain run diverges (ratio {c['ratio']:.0f})")
                continue
            fluid = t != W.SOLID
            row = dict(case=c, plain_steps=plain[0], plain_s=plain[1], plain_res=plain[2])
            msg = f"{S_test}^3 case {len(rows) + 1}: plain {plain[0]} updates {plain[1]:.2f} s (res {plain[2]:.1e})"
            # "warm": predicted densities and velocity; "warm_rho": predicted densities, fluid at rest
            for name, vel in variants:
                tw0 = time.perf_counter()
                init = warm_fields(net, c, S_test, velocity=vel)
                torch.cuda.synchronize()
                t_inf = time.perf_counter() - tw0
                warm = steps_to_steady(c, S_test, init, tol, check_every, max_steps)
                diff = max(float(np.abs(plain[3][k][0][fluid] - warm[3][k][0][fluid]).max()) for k in (0, 1))
                row.update({f"{name}_steps": warm[0], f"{name}_s": warm[1] + t_inf, f"{name}_res": warm[2],
                            f"{name}_infer_s": t_inf, f"{name}_max_density_diff": diff})
                msg += (f" | {name} {warm[0]} updates {warm[1] + t_inf:.2f} s (res {warm[2]:.1e}) "
                        f"max |d rho| {diff:.1e}")
            rows.append(row)
            log(msg)
        tests.append(dict(n=len(rows), size=S_test, tol=tol, check_every=check_every, max_steps=max_steps,
                          skipped_diverging=skipped, rows=rows))
    return dict(train=dict(n=n_train, kept=len(kept), size=S_train, gen_max_steps=gen_max_steps,
                           gen_residual_median=float(np.median(gres)), gen_s=t_gen, iters=iters, batch=batch,
                           train_s=t_train, tflops=flops / t_train / 1e12, loss=hist),
                tests=tests)


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="learned warm start: generate, train, compare steps to steady")
    ap.add_argument("--n-train", type=int, default=2000)
    ap.add_argument("--n-test", type=int, default=32)
    ap.add_argument("--n-test-large", type=int, default=8)
    ap.add_argument("--size-train", type=int, default=64)
    ap.add_argument("--test-sizes", default="64,128")
    ap.add_argument("--gen-max-steps", type=int, default=40000)
    ap.add_argument("--iters", type=int, default=2000)
    ap.add_argument("--tol", type=float, default=3e-6)
    ap.add_argument("--max-steps", type=int, default=60000)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    from . import build
    build.build()
    res = experiment(a.n_train, a.n_test, a.size_train, tuple(int(v) for v in a.test_sizes.split(",")),
                     a.gen_max_steps, a.iters, tol=a.tol, max_steps=a.max_steps, n_test_large=a.n_test_large)
    js = json.dumps(res, default=float)
    if a.out:
        open(a.out, "w").write(js)
    print(js)
