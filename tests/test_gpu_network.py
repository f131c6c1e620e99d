"""The warm-start U-Net on the GPU against an FP64 restatement built from the
convolution oracle.

The restatement rounds activations and gradients to BF16 at the same points
as the GPU path (so both sides see the same operands) and keeps everything
else in FP64.  Checked: the network output, the loss, and every layer's
weight and bias gradient.  Both sides round to BF16 at the same points, but a
value that the two accumulation orders put on different sides of a BF16
rounding boundary (or of a ReLU's zero) differs by one BF16 ulp, and these
differences compound through the 15 layers of the backward chain: measured
cosines run 0.997-0.9999 from launch to launch (the weight-gradient kernel
accumulates with atomics).  The bounds (cosine >= 0.99, relative L2 error
<= 15 %) sit below that spread; the test also shows they catch a wiring
mistake, by planting one (the channel order of the first skip
concatenation) in the restatement and requiring the GPU gradients to fail
against it.  The kernels themselves are checked one by one against the FP64
oracle to 2e-5.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_03254_gb300 import build
    build.build()
    from paper_1711_03254_gb300 import surrogate
    from oracle import conv
    conv.build()
    return torch, surrogate, conv


def _bf(torch, a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def test_network_gradients_match_fp64_restatement(env):
    torch, surrogate, conv = env
    S = 16
    net = surrogate.UNet3D(1, S, seed=3)
    rng = np.random.default_rng(9)
    x = rng.standard_normal((1, S, S, S, surrogate.CIN)).astype(np.float32)
    y = rng.standard_normal((1, S, S, S, surrogate.NOUT)).astype(np.float32) * 0.1
    m = (rng.random((1, S, S, S)) < 0.8).astype(np.uint8)
    wch = np.array([1.0, 10.0, 1.0, 1.0, 1.0], np.float32)
    dev = torch.device("cuda")
    out = net.forward(torch.from_numpy(x).to(dev)).cpu().numpy()
    loss = net.loss_and_grad(torch.from_numpy(y).to(dev), torch.from_numpy(m).to(dev), torch.from_numpy(wch).to(dev))
    net.backward()
    torch.cuda.synchronize()

    P = {n: dict(w=d["wb"].float().cpu().numpy().astype(np.float64), b=d["b"].cpu().numpy().astype(np.float64))
         for n, d in net.p.items()}
    bf = lambda a: _bf(torch, a)  # noqa: E731

    def fwd(name, inp, relu=True):
        o = conv.conv3d_fwd(inp, P[name]["w"], P[name]["b"])
        return bf(np.maximum(o, 0)) if relu else o

    def pool(a):
        n, s = a.shape[0], a.shape[1]
        return bf(a.reshape(n, s // 2, 2, s // 2, 2, s // 2, 2, -1).mean(axis=(2, 4, 6)))

    def up(a):
        return a.repeat(2, 1).repeat(2, 2).repeat(2, 3)

    def restate(swap_skip):
        c0, c1, c2, c3 = surrogate.LEVELS
        xb = bf(x)
        a0 = fwd("enc0a", xb)
        e0 = fwd("enc0b", a0)
        p1 = pool(e0)
        a1 = fwd("enc1a", p1)
        e1 = fwd("enc1b", a1)
        p2 = pool(e1)
        a2 = fwd("enc2a", p2)
        e2 = fwd("enc2b", a2)
        p3 = pool(e2)
        ab = fwd("bota", p3)
        b = fwd("botb", ab)
        cat2 = np.concatenate([up(b), e2], -1)
        d2a = fwd("dec2a", cat2)
        d2 = fwd("dec2b", d2a)
        cat1 = np.concatenate([up(d2), e1], -1)
        d1a = fwd("dec1a", cat1)
        d1 = fwd("dec1b", d1a)
        cat0 = np.concatenate([e0, up(d1)] if swap_skip else [up(d1), e0], -1)
        d0a = fwd("dec0a", cat0)
        d0 = fwd("dec0b", d0a)
        o = fwd("head", d0, relu=False)
        if not swap_skip:
            assert np.abs(out - o).max() < 2e-2 * np.abs(o).max()

        C = surrogate.NOUT
        cnt = o[..., :C].size
        dd = (o[..., :C] - y) * m[..., None]
        ref_loss = float((wch * dd * dd).sum() / cnt)
        if not swap_skip:
            assert abs(float(loss.item()) - ref_loss) < 2e-2 * ref_loss
        gout = np.zeros_like(o)
        gout[..., :C] = 2 * wch * dd / cnt
        gout = bf(gout)

        grads = {}

        def bwd(name, xin, gy, need_dx=True):
            dw, db = conv.conv3d_bwd_weight(xin, gy, P[name]["w"].shape[1])
            grads[name] = (dw, db)
            return bf(conv.conv3d_bwd_data(gy, P[name]["w"])) if need_dx else None

        def relu_b(act, g):
            return g * (act > 0)

        def up_b(g):
            n, s = g.shape[0], g.shape[1]
            return bf(g.reshape(n, s // 2, 2, s // 2, 2, s // 2, 2, -1).sum(axis=(2, 4, 6)))

        def pool_b_acc(g, old):
            return bf(old + g.repeat(2, 1).repeat(2, 2).repeat(2, 3) * 0.125)

        g_d0 = relu_b(d0, bwd("head", d0, gout))
        g_d0a = relu_b(d0a, bwd("dec0b", d0a, g_d0))
        g_cat0 = bwd("dec0a", cat0, g_d0a)
        g_d1 = relu_b(d1, up_b(g_cat0[..., c0:] if swap_skip else g_cat0[..., :c1]))
        g_d1a = relu_b(d1a, bwd("dec1b", d1a, g_d1))
        g_cat1 = bwd("dec1a", cat1, g_d1a)
        g_d2 = relu_b(d2, up_b(g_cat1[..., :c2]))
        g_d2a = relu_b(d2a, bwd("dec2b", d2a, g_d2))
        g_cat2 = bwd("dec2a", cat2, g_d2a)
        g_b = relu_b(b, up_b(g_cat2[..., :c3]))
        g_ab = relu_b(ab, bwd("botb", ab, g_b))
        g_p3 = bwd("bota", p3, g_ab)
        g_e2 = relu_b(e2, pool_b_acc(g_p3, g_cat2[..., c3:]))
        g_a2 = relu_b(a2, bwd("enc2b", a2, g_e2))
        g_p2 = bwd("enc2a", p2, g_a2)
        g_e1 = relu_b(e1, pool_b_acc(g_p2, g_cat1[..., c2:]))
        g_a1 = relu_b(a1, bwd("enc1b", a1, g_e1))
        g_p1 = bwd("enc1a", p1, g_a1)
        g_e0 = relu_b(e0, pool_b_acc(g_p1, g_cat0[..., :c0] if swap_skip else g_cat0[..., c1:]))
        g_a0 = relu_b(a0, bwd("enc0b", a0, g_e0))
        bwd("enc0a", xb, g_a0, need_dx=False)
        return grads

    def agree(grads):
        for name, d in net.p.items():
            gw = d["gw"].cpu().numpy().astype(np.float64).reshape(-1)
            gb = d["gb"].cpu().numpy().astype(np.float64)
            rw, rb = grads[name]
            rw = rw.reshape(-1)
            cos = float(gw @ rw / (np.linalg.norm(gw) * np.linalg.norm(rw) + 1e-300))
            ok = (cos >= 0.99 and np.linalg.norm(gw - rw) <= 0.15 * np.linalg.norm(rw)
                  and np.linalg.norm(gb - rb) <= 0.15 * np.linalg.norm(rb) + 1e-12)
            if not ok:
                return name, cos
        return None

    assert agree(restate(False)) is None
    # the same bounds reject a restatement with the skip channels swapped
    assert agree(restate(True)) is not None
