"""Learned warm start: a 3-D convolutional U-Net that maps a droplet-on-wall
problem (geometry, wettability, viscosity ratio, inclination, body force and
the plain initial droplet) to the steady fields of the two-component lattice
Boltzmann solver, trained on steady states the solver itself produces.

Every arithmetic step runs in this package's CUDA kernels (include/ws.h:
BF16 tensor-core convolutions with FP32 accumulation, pooling, upsampling,
ReLU, loss, Adam); PyTorch only provides device memory.  The network:

  level  resolution  channels   encoder            decoder (input = up(next) ++ skip)
    0       S          32       conv-conv          conv(64+32 -> 32)-conv
    1       S/2        64       pool-conv-conv     conv(96+64 -> 64)-conv
    2       S/4        96       pool-conv-conv     conv(128+96 -> 96)-conv
    3       S/8       128       pool-conv-conv     (bottom)
  3x3x3 convolutions with ReLU, a 1x1x1 head to 16 channels (5 used).

Input channels (16, 6 used): SOLID mask, cos(contact angle) on SOLID cells,
log10(viscosity ratio)/3, inclination/45 deg, body force * 1e4, plain initial
droplet indicator.  Output channels: phi = (rho1 - rho2)/rho, rho - 1,
100 * u_F (3).
"""
from __future__ import annotations

import math

import numpy as np

from . import ws

CIN = 16
COUT = 16
NOUT = 5
LEVELS = (32, 64, 96, 128)
U_SCALE = 100.0


class UNet3D:
    def __init__(self, batch: int, size: int, seed: int = 0):
        import torch
        if size % 8:
            raise ValueError("size must be a multiple of 8")
        self.torch = torch
        self.N, self.S = batch, size
        dev = torch.device("cuda")
        self.dev = dev
        c0, c1, c2, c3 = LEVELS
        # (name, Ci, Co, k)
        self.spec = [("enc0a", CIN, c0, 3), ("enc0b", c0, c0, 3),
                     ("enc1a", c0, c1, 3), ("enc1b", c1, c1, 3),
                     ("enc2a", c1, c2, 3), ("enc2b", c2, c2, 3),
                     ("bota", c2, c3, 3), ("botb", c3, c3, 3),
                     ("dec2a", c3 + c2, c2, 3), ("dec2b", c2, c2, 3),
                     ("dec1a", c2 + c1, c1, 3), ("dec1b", c1, c1, 3),
                     ("dec0a", c1 + c0, c0, 3), ("dec0b", c0, c0, 3),
                     ("head", c0, COUT, 1)]
        rng = np.random.default_rng(seed)
        self.p = {}
        for name, ci, co, k in self.spec:
            std = math.sqrt(2.0 / (k ** 3 * ci)) * (0.5 if name == "head" else 1.0)
            w = rng.standard_normal((co, k, k, k, ci)).astype(np.float32) * std
            d = dict(ci=ci, co=co, k=k,
                     w=torch.from_numpy(w).to(dev), b=torch.zeros(co, device=dev),
                     gw=torch.zeros_like(torch.from_numpy(w)).to(dev), gb=torch.zeros(co, device=dev),
                     mw=torch.zeros(w.size, device=dev), vw=torch.zeros(w.size, device=dev),
                     mb=torch.zeros(co, device=dev), vb=torch.zeros(co, device=dev),
                     wb=torch.from_numpy(w).to(dev).to(torch.bfloat16),
                     wf=torch.empty((ci, k, k, k, co), dtype=torch.bfloat16, device=dev))
            self.p[name] = d
        self.step_count = 0
        self._alloc(batch, size)

    # ------------------------------------------------------------------ buffers
    def _alloc(self, N, S):
        t = self.torch
        c0, c1, c2, c3 = LEVELS
        bf = dict(dtype=t.bfloat16, device=self.dev)

        def act(s, c):
            return t.empty((N, s, s, s, c), **bf)

        S1, S2, S3 = S // 2, S // 4, S // 8
        self.a = dict(x=act(S, CIN), a0=act(S, c0), cat0=act(S, c1 + c0), p1=act(S1, c0), a1=act(S1, c1),
                      cat1=act(S1, c2 + c1), p2=act(S2, c1), a2=act(S2, c2), cat2=act(S2, c3 + c2), p3=act(S3, c2),
                      ab=act(S3, c3), b=act(S3, c3), d2a=act(S2, c2), d2=act(S2, c2), d1a=act(S1, c1), d1=act(S1, c1),
                      d0a=act(S, c0), d0=act(S, c0))
        self.g = {k: t.empty_like(v) for k, v in self.a.items() if k != "x"}
        self.out = t.empty((N, S, S, S, COUT), dtype=t.float32, device=self.dev)
        self.gout = t.empty((N, S, S, S, COUT), **bf)

    # ------------------------------------------------------------------ pieces
    def _conv(self, name, x, y, relu=True):
        d = self.p[name]
        ws.ws_conv3d_fwd(x, d["wb"], d["b"], y, relu)

    def _conv_bwd(self, name, x, dy, dx):
        """Weight/bias gradients from (x, dy); input gradient into dx (if given)."""
        d = self.p[name]
        ws.ws_conv3d_bwd_weight(x, dy, d["gw"], d["gb"], d["k"])
        if dx is not None:
            ws.ws_conv3d_flip_weights(d["wb"], d["wf"])
            ws.ws_conv3d_fwd(dy, d["wf"], None, dx, False)

    # ------------------------------------------------------------------ forward / backward
    def forward(self, x_f32):
        """x_f32: FP32 [N, S, S, S, CIN] device tensor.  Returns FP32 [N, S, S, S, COUT]."""
        a = self.a
        c0, c1, c2, c3 = LEVELS
        ws.ws_to_bf16(x_f32, a["x"])
        e0, e1, e2 = a["cat0"][..., c1:], a["cat1"][..., c2:], a["cat2"][..., c3:]
        self._conv("enc0a", a["x"], a["a0"])
        self._conv("enc0b", a["a0"], e0)
        ws.ws_avgpool2(e0, a["p1"])
        self._conv("enc1a", a["p1"], a["a1"])
        self._conv("enc1b", a["a1"], e1)
        ws.ws_avgpool2(e1, a["p2"])
        self._conv("enc2a", a["p2"], a["a2"])
        self._conv("enc2b", a["a2"], e2)
        ws.ws_avgpool2(e2, a["p3"])
        self._conv("bota", a["p3"], a["ab"])
        self._conv("botb", a["ab"], a["b"])
        ws.ws_upsample2(a["b"], a["cat2"][..., :c3])
        self._conv("dec2a", a["cat2"], a["d2a"])
        self._conv("dec2b", a["d2a"], a["d2"])
        ws.ws_upsample2(a["d2"], a["cat1"][..., :c2])
        self._conv("dec1a", a["cat1"], a["d1a"])
        self._conv("dec1b", a["d1a"], a["d1"])
        ws.ws_upsample2(a["d1"], a["cat0"][..., :c1])
        self._conv("dec0a", a["cat0"], a["d0a"])
        self._conv("dec0b", a["d0a"], a["d0"])
        self._conv("head", a["d0"], self.out, relu=False)
        return self.out

    def backward(self):
        """Accumulates parameter gradients from self.gout (d loss / d out, BF16)."""
        a, g = self.a, self.g
        c0, c1, c2, c3 = LEVELS
        e0, e1, e2 = a["cat0"][..., c1:], a["cat1"][..., c2:], a["cat2"][..., c3:]
        ge0, ge1, ge2 = g["cat0"][..., c1:], g["cat1"][..., c2:], g["cat2"][..., c3:]
        self._conv_bwd("head", a["d0"], self.gout, g["d0"])
        ws.ws_relu_bwd(a["d0"], g["d0"])
        self._conv_bwd("dec0b", a["d0a"], g["d0"], g["d0a"])
        ws.ws_relu_bwd(a["d0a"], g["d0a"])
        self._conv_bwd("dec0a", a["cat0"], g["d0a"], g["cat0"])
        ws.ws_upsample2_bwd(g["cat0"][..., :c1], g["d1"])
        ws.ws_relu_bwd(a["d1"], g["d1"])
        self._conv_bwd("dec1b", a["d1a"], g["d1"], g["d1a"])
        ws.ws_relu_bwd(a["d1a"], g["d1a"])
        self._conv_bwd("dec1a", a["cat1"], g["d1a"], g["cat1"])
        ws.ws_upsample2_bwd(g["cat1"][..., :c2], g["d2"])
        ws.ws_relu_bwd(a["d2"], g["d2"])
        self._conv_bwd("dec2b", a["d2a"], g["d2"], g["d2a"])
        ws.ws_relu_bwd(a["d2a"], g["d2a"])
        self._conv_bwd("dec2a", a["cat2"], g["d2a"], g["cat2"])
        ws.ws_upsample2_bwd(g["cat2"][..., :c3], g["b"])
        ws.ws_relu_bwd(a["b"], g["b"])
        self._conv_bwd("botb", a["ab"], g["b"], g["ab"])
        ws.ws_relu_bwd(a["ab"], g["ab"])
        self._conv_bwd("bota", a["p3"], g["ab"], g["p3"])
        ws.ws_avgpool2_bwd(g["p3"], ge2, accumulate=True)
        ws.ws_relu_bwd(e2, ge2)
        self._conv_bwd("enc2b", a["a2"], ge2, g["a2"])
        ws.ws_relu_bwd(a["a2"], g["a2"])
        self._conv_bwd("enc2a", a["p2"], g["a2"], g["p2"])
        ws.ws_avgpool2_bwd(g["p2"], ge1, accumulate=True)
        ws.ws_relu_bwd(e1, ge1)
        self._conv_bwd("enc1b", a["a1"], ge1, g["a1"])
        ws.ws_relu_bwd(a["a1"], g["a1"])
        self._conv_bwd("enc1a", a["p1"], g["a1"], g["p1"])
        ws.ws_avgpool2_bwd(g["p1"], ge0, accumulate=True)
        ws.ws_relu_bwd(e0, ge0)
        self._conv_bwd("enc0b", a["a0"], ge0, g["a0"])
        ws.ws_relu_bwd(a["a0"], g["a0"])
        self._conv_bwd("enc0a", a["x"], g["a0"], None)

    def loss_and_grad(self, target, mask, wch):
        """Masked MSE of the first NOUT output channels; fills self.gout."""
        loss = self.torch.zeros(1, dtype=self.torch.float32, device=self.dev)
        ws.ws_mse_loss(self.out, target, mask, wch, self.gout, loss)
        return loss

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step_count += 1
        t = self.step_count
        lr_t = lr * math.sqrt(1 - beta2 ** t) / (1 - beta1 ** t)
        for name, d in self.p.items():
            ws.ws_adam(d["w"], d["mw"], d["vw"], d["gw"], d["wb"], lr_t, beta1, beta2, eps)
            ws.ws_adam(d["b"], d["mb"], d["vb"], d["gb"], None, lr_t, beta1, beta2, eps)

    def flops_per_sample(self) -> float:
        """Multiply-adds x 2 of the convolutions in one forward pass of one sample."""
        S = self.S
        res = {"enc0": S, "enc1": S // 2, "enc2": S // 4, "bot": S // 8, "dec2": S // 4, "dec1": S // 2,
               "dec0": S, "head": S}
        tot = 0.0
        for name, ci, co, k in self.spec:
            s = res[name[:-1] if name != "head" else "head"]
            tot += 2.0 * s ** 3 * k ** 3 * ci * co
        return tot


# ---------------------------------------------------------------------- problem encoding

def encode_inputs(cell_type, theta_deg, nu_ratio, incline_deg, body_force, rho2_init):
    """FP32 [S, S, S, CIN] network input of one case (see module docstring)."""
    S = cell_type.shape[0]
    x = np.zeros((S, S, S, CIN), np.float32)
    solid = cell_type == 1
    x[..., 0] = solid
    x[..., 1] = np.where(solid, math.cos(math.radians(theta_deg)), 0.0)
    x[..., 2] = math.log10(nu_ratio) / 3.0
    x[..., 3] = incline_deg / 45.0
    x[..., 4] = body_force * 1e4
    x[..., 5] = np.where(solid, 0.0, rho2_init)
    return x


def encode_targets(rho1, rho2, u):
    """FP32 [S, S, S, NOUT] training target from the steady fields."""
    rho = rho1 + rho2
    safe = np.where(rho > 0, rho, 1.0)
    y = np.zeros(rho1.shape + (NOUT,), np.float32)
    y[..., 0] = np.where(rho > 0, (rho1 - rho2) / safe, 0.0)
    y[..., 1] = np.where(rho > 0, rho - 1.0, 0.0)
    y[..., 2:5] = u * U_SCALE
    return y


def decode_fields(out, cell_type):
    """Network output [S, S, S, >=NOUT] -> (rho1, rho2, u) for lbm_set_fields."""
    phi = np.clip(out[..., 0], -1.0, 1.0)
    rho = np.maximum(1.0 + out[..., 1], 0.05)
    rho1 = 0.5 * rho * (1.0 + phi)
    rho2 = 0.5 * rho * (1.0 - phi)
    u = out[..., 2:5] / U_SCALE
    solid = cell_type == 1
    rho1[solid] = 0.0
    rho2[solid] = 0.0
    u[solid] = 0.0
    return rho1.astype(np.float64), rho2.astype(np.float64), u.astype(np.float64)
