"""Benchmark: MLUPS and fraction of the HBM roofline of the two-component
Shan-Chen D3Q19 update on one GB300.

Workload: random packed spheres 256^3 (overlapping spheres r = 12 to porosity
0.40, seed 3), 1 % minority component as droplets r = 4, kinematic viscosities
1.0 / 0.01 (ratio 100), G = -2.2, rho^s = 0, body force 1e-6 along x, wall
model 2, FP32 arithmetic, storage selected by --precision (default 16-bit
shifted).  A step is one update of the whole domain.  f (>= 1.27 GB) is larger
than L2, so no flush is needed between steps.

The roofline object is for the dominant kernel of the step: the method's
algorithmic bytes per fluid-cell update (f read once and written once, 38
values each way per component pair, plus the cell-type byte: 76 s + 1 for
storage size s) times the fluid cells, over the kernel's average launch time,
taken with CUDA events around every launch on the launching stream during the
timed region (lbm_timing_begin / lbm_timing_end).  `step_frac` puts the same
bytes over the whole step, and `kernel_impl_frac` puts the bytes the dominant
kernel itself must move in this design over its launch time.

Other workloads (--workload): "droplet" (all-fluid periodic box), "rough"
(the rough channel 2n x n x n with an invading slug), "sweep" (16 instances of
the two-layer channel 4 x 128 x 4, viscosity ratios to 1000, batched in one
context: AUTO steps them in one persistent launch).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp16s|bf16s]
                  [--workload spheres|droplet|rough|sweep] [--kernel auto|compact|...]
  python bench.py --impl reference ...   (the FP64 CPU oracle on host cores)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 256
NU = (1.0, 0.01)  # majority / minority kinematic viscosity (ratio 100)
G = -2.2


def params(nu=NU, G=G):
    return dict(tau=(nu[0] * 3 + 0.5, nu[1] * 3 + 0.5), G=G, rho_s=0.0, g=(1e-6, 0.0, 0.0))


PARAMS = params()
# all-fluid droplet check case: tau = 1 for both components (nu = 1/6)
DROPLET_PARAMS = params(nu=(1 / 6, 1 / 6))
# rough channel 512 x 256 x 256: defending component 1 at nu = 1.7, invading
# component 2 at nu = 0.0017 (ratio 1000), wetting walls (rho^s = 0.2 favours
# the invading component), periodic ends driven by a body force of 1e-5 along x
ROUGH_PARAMS = dict(tau=(1.7 * 3 + 0.5, 0.0017 * 3 + 0.5), G=G, rho_s=0.2, g=(1e-5, 0.0, 0.0))
WORKLOAD_PARAMS = {"spheres": PARAMS, "droplet": DROPLET_PARAMS, "rough": ROUGH_PARAMS}
F_BYTES = {"fp64": 8, "fp32": 4, "fp16s": 2, "bf16s": 2}


def alg_bytes_per_cell(part: str, precision: str) -> int:
    """Bytes one fluid-cell update of `part` must move at least: every array
    element it needs read once and every result written once.
      f: 2 components x 19 directions x storage bytes, read (and written);
      psi: 2 values of the arithmetic type; link word 4 B; cell-list entry 4 B;
      reference densities (shifted storage): 2 x FP16 read, and written with f."""
    s = F_BYTES[precision]
    t = 8 if precision == "fp64" else 4
    ref = 0 if precision == "fp64" else 4
    if part == "psi":
        return 38 * s + 4 + 4 + ref + 2 * t
    if part == "collide":
        return 76 * s + 4 + 4 + 2 * t + 2 * ref
    if part == "fused_compact":
        # f once each way, reference pairs, packed coordinates and geometry word;
        # psi stays on chip
        return 76 * s + 4 + 4 + 2 * ref
    if part == "persistent":
        # each update of the persistent launch: both passes of the compact update
        return alg_bytes_per_cell("psi", precision) + alg_bytes_per_cell("collide", precision)
    return 76 * s + 4 + 2 * ref  # fused, and each update of a cluster launch
# DRAM traffic of the dominant kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of a launch / its fluid cells),
# keyed by kernel/precision/workload, with the hash of the source files the
# kernel is built from at the time of the capture; any change of them voids it.
COMPACT_SOURCES = ["lbm_types.h", "lbm_device.cuh", "lbm_pair2.cuh", "lbm_compact.cuh", "lbm_compact_update.cuh"]
DENSE_SOURCES = ["lbm_types.h", "lbm_device.cuh", "lbm_twopass.cuh"]
NCU_TRAFFIC = {
    # 128^3 packed spheres (837,994 non-solid cells), dense layout, ncu --set full:
    # 273.1 MB read + 103.1 MB written in one launch
    "k_collide/fp16s/spheres": {"bytes_per_fluid_cell": 449.0, "src": "cad4ff68f880e7db", "files": DENSE_SOURCES,
                                "how": "ncu --set full, one launch at 128^3, scaled by non-solid cells"},
    # the benchmark itself (256^3, 6,710,661 non-solid cells), one launch each,
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum:
    #   k_collide_c2: 649,660,672 B read + 497,568,000 B written = 171.0 B per cell
    #   k_psi_c:      595,477,504 B read +  50,510,080 B written =  96.3 B per cell
    "k_collide_c2/fp16s/spheres": {"bytes_per_fluid_cell": 170.96, "src": "856ecc299163ec5a",
                                   "files": COMPACT_SOURCES, "step_bytes_per_fluid_cell": 170.96 + 96.26,
                                   "how": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch at 256^3"},
}
# FP64 mode is bound by the FP64 pipe.  Executed FP64 flops per non-solid cell
# (DADD + DMUL + 2 DFMA from ncu, 128^3 packed spheres, eq_order 0) and the
# FP64 peak: 2 DFMA per clock per SM (152 SMs, 2.07 GHz) = 1.26 TFLOP/s.
# (Counted on sources 4ac21a08ce947105; the next change of these files touched
# only the psi pass, so the FP64 update's code is the one counted.)
FP64_FLOPS = {"k_collide_c": {"flops_per_fluid_cell": 813.7, "src": "1f62a0de098d92be", "files": COMPACT_SOURCES}}
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12


E2E_SAMPLES = 3


def sources_hash(files=COMPACT_SOURCES) -> str:
    h = hashlib.sha256()
    for s in files:
        p = os.path.join(ROOT, "paper_1711_03254_gb300", "csrc", s)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def workload(n=N, kind="spheres"):
    """The packed-sphere benchmark geometry n^3; (kind="droplet") an all-fluid
    periodic box with one droplet of radius n/8, used to see the kernel without
    SOLID cells; (kind="rough") the rough channel 2n x n x n with periodic ends
    and an invading slug of component 2 in its first 32 planes."""
    from paper_1711_03254_gb300 import workloads as W
    if kind == "droplet":
        return W.droplet(n, n, n, n / 8.0)
    if kind == "rough":
        return W.rough_channel(2 * n, n, n, seed=4, invaded_length=32, ends="periodic")
    # the generated geometry is cached under a name that carries a hash of the
    # generator's source, so an edited generator never reuses an old file
    gen = os.path.join(ROOT, "paper_1711_03254_gb300", "workloads.py")
    tag = hashlib.sha256(open(gen, "rb").read()).hexdigest()[:12]
    cache = os.path.join(tempfile.gettempdir(), f"lbm_spheres_{n}_{tag}.npz")
    if os.path.exists(cache):
        z = np.load(cache)
        return z["t"], z["r1"], z["r2"], z["u"]
    t, r1, r2, u = W.packed_spheres(n=n, r=12.0, porosity=0.40, seed=3, droplet_r=4.0, minority=0.01)
    try:
        np.savez(cache, t=t, r1=r1, r2=r2, u=u)
    except OSError:
        pass
    return t, r1, r2, u


# the layered-channel viscosity sweep: 16 instances of 4 x 128 x 4 (walls at
# y), viscosity ratio {1, 10, 100, 1000} with the minimum nu 0.0017, the
# low-viscosity component along the walls or in the core, layouts 1|2|1 and
# 1|2.  G = -1.8: with both components at nu 0.0017 the layers are unstable at
# -2.2 (in the oracle too).  Body force 4e-8: at 1e-6 the nu = 0.0017 layers
# would flow at about the lattice sound speed.
SWEEP_G, SWEEP_FORCE = -1.8, 4e-8


def sweep_cases():
    cases = []
    for ratio in (1, 10, 100, 1000):
        for low_at_wall in (True, False):
            for layout in ("121", "12"):
                lo, hi = 0.0017, 0.0017 * ratio
                cases.append((layout,) + ((lo, hi) if low_at_wall else (hi, lo)))
    return cases


def batch_workload(n, kind):
    """(cell types, rho1, rho2, u with a leading instance axis, the instances'
    parameters) of a bench workload; every workload but the sweep is one
    instance."""
    if kind == "sweep":
        from paper_1711_03254_gb300 import workloads as W
        ts, a, b, v, ps = [], [], [], [], []
        for layout, nu1, nu2 in sweep_cases():
            t, r1, r2, u = W.layered_channel(4, 128, 4, layout=layout, wall_comp_nu=nu1, core_comp_nu=nu2,
                                             g=SWEEP_FORCE)
            ts.append(t), a.append(r1), b.append(r2), v.append(u)
            ps.append(dict(tau=(nu1 * 3 + 0.5, nu2 * 3 + 0.5), G=SWEEP_G, g=(SWEEP_FORCE, 0.0, 0.0)))
        return np.stack(ts), np.stack(a), np.stack(b), np.stack(v), ps
    t, r1, r2, u = workload(n, kind)
    return t[None], r1[None], r2[None], u[None], [WORKLOAD_PARAMS[kind]]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index: int):
        self.path = f"/tmp/lbm_clocks_{os.getpid()}.csv"
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "samples": len(rows), "reasons": sorted(reasons)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    from paper_1711_03254_gb300 import replicas
    return replicas.max_over_ranks(x)


def cpu_baseline(t, r1, r2, u, target_s=15.0, crop=64, params=None, name="256^3 packed-sphere workload"):
    """Time the FP64 oracle, as it stands, on host cores over a bounded sample:
    a crop^3 corner of the same geometry for as many updates as fit ~target_s."""
    import oracle
    oracle.build()
    c = (slice(0, crop),) * 3
    tc, a, b, v = t[c].copy(), r1[c].copy(), r2[c].copy(), u[c].copy()
    sim = oracle.OracleSim(crop, crop, crop, [params or PARAMS])
    sim.set_geometry(tc[None])
    sim.set_fields(a[None], b[None], v[None])
    sim.step(1)
    t0 = time.perf_counter()
    sim.step(2)
    per = (time.perf_counter() - t0) / 2
    steps = max(1, int(target_s / max(per, 1e-6)))
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    fluid = int((tc != 1).sum())
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": fluid * steps / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{crop}^3 corner of the {name}, {steps} updates, FP64"}


def cpu_baseline_batch(t, r1, r2, u, params, name, target_s=15.0):
    """The FP64 oracle over all instances of a small batched workload, for
    as many updates as fit ~target_s."""
    import oracle
    oracle.build()
    B, nz, ny, nx = t.shape
    sim = oracle.OracleSim(nx, ny, nz, params)
    sim.set_geometry(t)
    sim.set_fields(r1, r2, u)
    sim.step(1)
    t0 = time.perf_counter()
    sim.step(2)
    per = (time.perf_counter() - t0) / 2
    steps = max(1, int(target_s / max(per, 1e-6)))
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    fluid = int((t != 1).sum())
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": fluid * steps / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"the {name}, all instances, {steps} updates, FP64"}


def run_reference(args):
    # rank 0 alone times the oracle; the other ranks leave without work (no
    # process group is needed for that)
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle
    oracle.build()
    t, r1, r2, u = workload()
    crop = 64
    c = (slice(0, crop),) * 3
    tc = t[c].copy()
    fluid = int((tc != 1).sum())
    sim = oracle.OracleSim(crop, crop, crop, [PARAMS])
    sim.set_geometry(tc[None])
    sim.set_fields(r1[c].copy()[None], r2[c].copy()[None], u[c].copy()[None])
    sim.step(1)
    t0 = time.perf_counter()
    sim.step(2)
    per = (time.perf_counter() - t0) / 2
    # W untimed warm-up samples, then K timed samples, each a run of updates of
    # the same crop sized so that the whole run stays near two minutes
    for _ in range(args.warmup):
        sim.step(max(1, int(min(2.0, 20.0 / max(1, args.warmup)) / max(per, 1e-6))))
    target = min(20.0, 120.0 / max(1, args.steps))
    n = max(1, int(target / max(per, 1e-6)))
    rates, times = [], []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        sim.step(n)
        dt = time.perf_counter() - t0
        rates.append(fluid * n / dt / 1e6)
        times.append(dt / n * 1e3)
    v = statistics.median(rates)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    cb = {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
          "sample": (f"{len(rates)} timed samples of {n} updates each on the {crop}^3 corner of the 256^3 "
                     f"packed-sphere workload, FP64 (median rate)")}
    line = {"impl": "reference", "metric": "MLUPS (fluid-cell updates per second, 2-comp D3Q19)", "value": v,
            "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(statistics.median(times), 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "packed spheres 256^3 (sampled as 64^3 corner on host cores)",
                       "precision": "fp64", "ms_per_step": "one update of the 64^3 sample"},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                                          "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--precision", default="fp16s", choices=["fp32", "fp16s", "bf16s", "fp64"])
    ap.add_argument("--kernel", default="auto")
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--size", type=int, default=N)
    ap.add_argument("--workload", default="spheres", choices=["spheres", "droplet", "rough", "sweep"])
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    from paper_1711_03254_gb300 import build, lbm
    build.build()
    lbm.use_torch_allocator()
    n = args.size
    t, r1, r2, u, params = batch_workload(n, args.workload)
    nz, ny, nx = t.shape[1:]
    fluid = int((t != 1).sum())  # non-solid cells of all instances
    stream = torch.cuda.current_stream()

    sim = lbm.Sim(nx, ny, nz, params, precision=args.precision, kernel=args.kernel)
    lbm.lbm_set_stream(sim.ctx, stream.cuda_stream)
    sim.set_geometry(t)
    sim.set_fields(r1, r2, u)
    sim.step(args.warmup)
    torch.cuda.synchronize()
    red0 = sim.reduce(allow_diverged=True)

    clk = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    l0 = sim.launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lbm.lbm_timing_begin(sim.ctx, 2 * args.steps + 2)
    ev0.record(stream)
    sim.step(args.steps)
    ev1.record(stream)
    timing = lbm.lbm_timing_end(sim.ctx)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = clk.stop()
    launches = sim.launches - l0
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms, ws)
    red1 = sim.reduce(allow_diverged=True)
    mass_drift = float(np.max(np.abs(red1[:, :2] - red0[:, :2]) / red0[:, :2]))

    mlups = fluid * args.steps * ws / (ms_max / 1e3) / 1e6
    hbm, peak_kind = peaks()
    # the dominant kernel of the step: largest summed event time
    part = max(timing, key=lambda k: timing[k][0])
    part_ms, part_launches = timing[part]
    strategy = lbm.lbm_resolved_kernel(sim.ctx, args.steps)
    kernel_name = {"psi": "k_psi", "collide": "k_collide", "fused": "k_fused", "cluster": "k_cluster"}[part]
    if strategy == "persistent":
        kernel_name = "k_persist_c"
    if strategy == "compact":
        # compact layout: packed-pair update for the FP32-arithmetic storages
        kernel_name += {"psi": "_c", "collide": "_c" if args.precision == "fp64" else "_c2"}[part]
    if strategy == "fused_compact":
        kernel_name = "k_fused_c"
    # the method's own bytes per fluid-cell update (f in + f out + type byte):
    # the roofline's algorithmic figure for the dominant kernel and the step
    method_bytes = 2 * 38 * F_BYTES[args.precision] + 1
    # what this kernel moves at least
    impl_bytes = alg_bytes_per_cell("fused_compact" if strategy == "fused_compact" else
                                    ("persistent" if strategy == "persistent" else part), args.precision)
    updates_per_launch = args.steps if part == "cluster" else 1
    avg_s = part_ms / part_launches / 1e3
    achieved = method_bytes * fluid * updates_per_launch / avg_s / 1e9
    key = f"{kernel_name}/{args.precision}/{args.workload}"
    tr = NCU_TRAFFIC.get(key)
    traffic = None
    if tr and tr.get("src") == sources_hash(tr["files"]):
        traffic = round(tr["bytes_per_fluid_cell"] * fluid * updates_per_launch)
    step_s = (ms / args.steps) / 1e3
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": traffic, "peak_kind": peak_kind,
            "traffic_source": tr.get("how") if traffic is not None else None,
            "kernel": kernel_name, "algorithmic_bytes_per_fluid_cell": method_bytes,
            "avg_launch_ms": round(avg_s * 1e3, 4), "launches": part_launches,
            "share_of_step": round(part_ms / ms, 4),
            "parts_ms": {k: round(v[0] / v[1], 4) for k, v in timing.items()},
            # the whole step (every kernel of an update) on the method's bytes
            "step_frac": round(method_bytes * fluid / step_s / 1e9 / hbm, 4),
            # the dominant kernel on the bytes it must move in this design
            # (psi, coordinates, links, reference densities besides f)
            "kernel_impl_bytes_per_fluid_cell": impl_bytes,
            "kernel_impl_frac": round(impl_bytes * fluid * updates_per_launch / avg_s / 1e9 / hbm, 4)}
    if tr and traffic is not None:
        # measured DRAM bytes of one step over the method's bytes
        step_tr = tr.get("step_bytes_per_fluid_cell")
        if step_tr:
            roof["step_traffic_bytes_per_fluid_cell"] = step_tr
            roof["wasted_traffic_ratio"] = round(step_tr / method_bytes, 3)

    fl = FP64_FLOPS.get(kernel_name)
    if args.precision == "fp64" and fl and fl["src"] == sources_hash(fl["files"]):
        # FP64 arithmetic: the FP64 pipe, not HBM, bounds the update
        tf = fl["flops_per_fluid_cell"] * fluid * updates_per_launch / avg_s / 1e12
        roof.update({"bound": "alu", "achieved": round(tf, 4), "peak": round(FP64_PEAK_TFLOPS, 3),
                     "unit": "TFLOP/s", "frac": round(tf / FP64_PEAK_TFLOPS, 4),
                     "peak_kind": "derived: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz",
                     "flops_per_fluid_cell": fl["flops_per_fluid_cell"]})

    # end to end through the C ABI with host buffers: a fresh context per
    # sample, the median of E2E_SAMPLES samples (the host<->device copies of a
    # shared host occasionally take several times their usual 3-4 ms)
    e2e = None
    if ws == 1:
        ke = max(1, min(args.steps, 100))

        def pinned(a):
            # page-locked host array (the copies then run as DMA from/to it)
            dt_ = {np.dtype(np.float64): torch.float64, np.dtype(np.uint8): torch.uint8}[a.dtype]
            return torch.empty(a.shape, dtype=dt_, pin_memory=True).numpy()
        th, r1h, r2h, uh = pinned(t), pinned(r1), pinned(r2), pinned(u)
        th[...], r1h[...], r2h[...], uh[...] = t, r1, r2, u
        r1b, r2b, ub = pinned(r1), pinned(r2), pinned(u)
        rates = []
        for _ in range(E2E_SAMPLES):
            sim2 = lbm.Sim(nx, ny, nz, params, precision=args.precision, kernel=args.kernel)
            lbm.lbm_set_stream(sim2.ctx, stream.cuda_stream)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lbm.lbm_set_geometry(sim2.ctx, th)
            lbm.lbm_set_fields(sim2.ctx, r1h, r2h, uh)
            sim2.step(ke)
            lbm.lbm_get_fields(sim2.ctx, r1b, r2b, ub)
            dt = time.perf_counter() - t0
            rates.append(fluid * ke / dt / 1e6)
            sim2.close()
        h2d = t.size * 1 + r1.size * 8 * 2 + u.size * 8
        d2h = r1.size * 8 * 2 + u.size * 8
        e2e = {"value": round(float(np.median(rates)), 1), "unit": "MLUPS", "steps": ke,
               "h2d_bytes_per_step": h2d // ke, "d2h_bytes_per_step": d2h // ke, "host_buffers": "pinned",
               "samples": [round(v, 1) for v in rates], "stat": "median"}

    cb = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        if args.workload == "sweep":
            cb = cpu_baseline_batch(t, r1, r2, u, params, "16-instance layered-channel sweep 4x128x4")
        else:
            cb = cpu_baseline(t[0], r1[0], r2[0], u[0], params=params[0],
                              name={"spheres": f"{n}^3 packed-sphere workload",
                                    "droplet": f"{n}^3 droplet workload",
                                    "rough": f"{2 * n}x{n}x{n} rough channel"}[args.workload])

    if rank == 0:
        line = {"metric": "MLUPS (fluid-cell updates per second, 2-comp D3Q19)", "value": round(mlups, 1),
                "unit": "MLUPS", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
                "config": {"workload": {
                    "spheres": (f"packed spheres {n}^3, r=12, porosity 0.40, 1% minority r=4, "
                                f"nu {NU[0]}/{NU[1]} (ratio 100), G={G}, g=1e-6, wall model 2"),
                    "droplet": f"periodic droplet {n}^3, R={n // 8}, tau 1/1, G={G}, no walls",
                    "rough": (f"rough channel {2 * n}x{n}x{n}, walls on y and z with seeded bumps <= 4, "
                              f"periodic ends, invading slug nu 0.0017 vs defending nu 1.7 (ratio 1000), "
                              f"G={G}, rho^s 0.2, g=1e-5 along x, wall model 2"),
                    "sweep": (f"viscosity sweep: 16 instances of the two-layer channel 4x128x4 (walls at y), "
                              f"ratio 1/10/100/1000 with min nu 0.0017, low viscosity at the walls or in the "
                              f"core, layouts 1|2|1 and 1|2, G={SWEEP_G}, g={SWEEP_FORCE}, "
                              f"batched in one context")}[args.workload],
                           "storage": args.precision, "kernel": args.kernel, "strategy": strategy,
                           "fluid_cells": fluid,
                           "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{ws}"},
                "roofline": roof, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clocks, "mass_drift": mass_drift}
        print(json.dumps(line))
    sim.close()


if __name__ == "__main__":
    main()
