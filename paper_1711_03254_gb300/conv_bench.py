"""Throughput of the surrogate's convolutions, layer by layer.

    python -m paper_1711_03254_gb300.conv_bench [--size 64] [--batch 4] [--reps 20]

For every 3x3x3 layer of the U-Net (surrogate.Surrogate's layer table at the
given resolution and batch) this times, with CUDA events on the current stream
after warm-up:
  - the forward convolution with each forward kernel ("resident": the
    automatic resident choice, "pertile": one block per tile, "persistent":
    persistent wherever it fits, "gather": the gathered kernel);
  - the data gradient (the forward kernel on flipped weights, Ci and Co
    exchanged; the first layer has none);
  - the weight gradient with each of its kernels ("resident": the automatic
    resident choice, "pairs": tap-pair rows only, "gather").
It prints one JSON line per layer and a summary line.  TFLOP/s counts
2 Ci Co 27 multiply-adds per output position; `frac` divides by the measured
BF16 tensor peak of MEASURED_PEAKS.json when that file is present.  Inputs are
random BF16 values; the layers are compute-bound, so launches are timed back
to back without flushing L2.  A last line times whole training iterations
(--train-iters).
"""
from __future__ import annotations

import argparse
import json
import os


def _peak():
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    for key in ("bf16_tflops", "bf16_dense_tflops"):
        if isinstance(d.get(key), (int, float)):
            return float(d[key])
    return None


def _time(torch, fn, reps):
    for _ in range(3):
        fn()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps  # ms


def layers(size: int):
    from .surrogate import LEVELS, CIN
    c0, c1, c2, c3 = LEVELS
    res = {0: size, 1: size // 2, 2: size // 4, 3: size // 8}
    spec = [("enc0a", CIN, c0, 0), ("enc0b", c0, c0, 0), ("enc1a", c0, c1, 1), ("enc1b", c1, c1, 1),
            ("enc2a", c1, c2, 2), ("enc2b", c2, c2, 2), ("bota", c2, c3, 3), ("botb", c3, c3, 3),
            ("dec2a", c3 + c2, c2, 2), ("dec2b", c2, c2, 2), ("dec1a", c2 + c1, c1, 1), ("dec1b", c1, c1, 1),
            ("dec0a", c1 + c0, c0, 0), ("dec0b", c0, c0, 0)]
    return [(name, ci, co, res[lvl]) for name, ci, co, lvl in spec]


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--size", type=int, default=64)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--train-iters", type=int, default=50,
                    help="also time this many whole training iterations (0: skip)")
    args = ap.parse_args(argv)
    import torch
    from . import build
    build.build()
    from . import ws
    dev = torch.device("cuda:0")
    g = torch.Generator(device=dev)
    g.manual_seed(1)
    peak = _peak()
    tot = {"fwd_resident": 0.0, "fwd_pertile": 0.0, "fwd_persistent": 0.0, "fwd_gather": 0.0,
           "bwd_data": 0.0, "bwd_weight_resident": 0.0, "bwd_weight_pairs": 0.0, "bwd_weight_gather": 0.0}
    flops_tot = {"fwd": 0.0, "bwd_data": 0.0, "bwd_weight": 0.0}
    for name, ci, co, s in layers(args.size):
        N = args.batch
        x = torch.randn((N, s, s, s, ci), generator=g, device=dev).to(torch.bfloat16)
        w = (torch.randn((co, 3, 3, 3, ci), generator=g, device=dev) * 0.05).to(torch.bfloat16)
        b = torch.zeros(co, device=dev)
        y = torch.empty((N, s, s, s, co), dtype=torch.bfloat16, device=dev)
        dy = torch.randn((N, s, s, s, co), generator=g, device=dev).to(torch.bfloat16)
        dx = torch.empty((N, s, s, s, ci), dtype=torch.bfloat16, device=dev)
        wf = torch.empty((ci, 3, 3, 3, co), dtype=torch.bfloat16, device=dev)
        ws.ws_conv3d_flip_weights(w, wf)
        gw = torch.zeros((co, 3, 3, 3, ci), dtype=torch.float32, device=dev)
        gb = torch.zeros(co, dtype=torch.float32, device=dev)
        flops = 2.0 * N * s ** 3 * 27 * ci * co
        row = dict(layer=name, size=s, batch=N, Ci=ci, Co=co, gflop=round(flops / 1e9, 2))
        prev = ws.ws_conv3d_fwd_algo("auto")
        prev_w = ws.ws_conv3d_bwd_weight_algo("auto")
        try:
            for algo in ("resident", "pertile", "persistent", "gather"):
                ws.ws_conv3d_fwd_algo(algo)
                ms = _time(torch, lambda: ws.ws_conv3d_fwd(x, w, b, y, True), args.reps)
                row[f"fwd_{algo}_ms"] = round(ms, 4)
                row[f"fwd_{algo}_tflops"] = round(flops / ms / 1e9, 1)
                tot[f"fwd_{algo}"] += ms
            ws.ws_conv3d_fwd_algo("auto")
            if name != "enc0a":
                ms = _time(torch, lambda: ws.ws_conv3d_fwd(dy, wf, None, dx, False), args.reps)
                row["bwd_data_ms"] = round(ms, 4)
                row["bwd_data_tflops"] = round(flops / ms / 1e9, 1)
                tot["bwd_data"] += ms
                flops_tot["bwd_data"] += flops
            for algo in ("resident", "pairs", "gather"):
                ws.ws_conv3d_bwd_weight_algo(algo)
                ms = _time(torch, lambda: ws.ws_conv3d_bwd_weight(x, dy, gw, gb, 3), args.reps)
                row[f"bwd_weight_{algo}_ms"] = round(ms, 4)
                row[f"bwd_weight_{algo}_tflops"] = round(flops / ms / 1e9, 1)
                tot[f"bwd_weight_{algo}"] += ms
        finally:
            ws.ws_conv3d_fwd_algo(prev)
            ws.ws_conv3d_bwd_weight_algo(prev_w)
        flops_tot["fwd"] += flops
        flops_tot["bwd_weight"] += flops
        if peak:
            row["fwd_resident_frac"] = round(row["fwd_resident_tflops"] / peak, 3)
        print(json.dumps(row), flush=True)
    if ws.ws_tc_status() != 0:
        raise RuntimeError("a tensor-core convolution gave up on a bounded wait")
    summ = dict(summary=True, size=args.size, batch=args.batch, peak_bf16_tflops=peak)
    for key, ms in tot.items():
        kind = "fwd" if key.startswith("fwd") else ("bwd_weight" if key.startswith("bwd_weight") else key)
        fl = flops_tot[kind]
        summ[f"{key}_ms"] = round(ms, 3)
        summ[f"{key}_tflops"] = round(fl / ms / 1e9, 1)
        if peak:
            summ[f"{key}_frac"] = round(fl / ms / 1e9 / peak, 3)
    print(json.dumps(summ), flush=True)
    if args.train_iters > 0:
        print(json.dumps(train_step(torch, args.size, args.batch, args.train_iters, peak)), flush=True)


def train_step(torch, size, batch, iters, peak):
    """Whole training iterations of the U-Net (BF16 cast, forward, masked loss,
    backward, Adam) on random inputs, as the warm-start training runs them, with
    the automatic kernel choice and with the gathered kernels; TFLOP/s counts
    the convolutions' 3 x forward multiply-adds."""
    from . import surrogate
    dev = torch.device("cuda:0")
    g = torch.Generator(device=dev)
    g.manual_seed(2)
    net = surrogate.UNet3D(batch, size, seed=0)
    shape = (batch, size, size, size)
    x = torch.randn(shape + (surrogate.CIN,), generator=g, device=dev)
    y = torch.randn(shape + (surrogate.NOUT,), generator=g, device=dev)
    m = torch.ones(shape, dtype=torch.uint8, device=dev)
    wch = torch.ones(surrogate.NOUT, dtype=torch.float32, device=dev)

    def it():
        net.forward(x)
        net.loss_and_grad(y, m, wch)
        net.backward()
        net.adam_step(lr=1e-4)

    from . import ws
    fl = 3.0 * net.flops_per_sample() * batch
    out = dict(train=True, size=size, batch=batch, iters=iters)
    prev = ws.ws_conv3d_fwd_algo("auto"), ws.ws_conv3d_bwd_weight_algo("auto")
    try:
        for algo in ("auto", "gather"):
            ws.ws_conv3d_fwd_algo(algo)
            ws.ws_conv3d_bwd_weight_algo(algo)
            ms = _time(torch, it, iters)
            out[f"{algo}_ms_per_iter"] = round(ms, 3)
            out[f"{algo}_tflops"] = round(fl / ms / 1e9, 1)
            if peak:
                out[f"{algo}_frac"] = round(fl / ms / 1e9 / peak, 3)
    finally:
        ws.ws_conv3d_fwd_algo(prev[0])
        ws.ws_conv3d_bwd_weight_algo(prev[1])
    return out


if __name__ == "__main__":
    main()
