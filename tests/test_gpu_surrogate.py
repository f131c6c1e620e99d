"""Surrogate kernels on the GPU against the FP64 oracle (convolutions) and
plain NumPy restatements (pooling, upsampling, ReLU, loss, Adam).

Operands are rounded to BF16 on the host first, so both sides multiply the
same numbers; the GPU accumulates in FP32 and the bound is relative to the
largest output: 2e-5 for the convolutions (FP32 sums of <= 27 * 224 exact
products), 1e-2 where a BF16 result is stored.
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
    from paper_1711_03254_gb300 import ws
    from oracle import conv
    conv.build()
    return torch, ws, conv


def _bf16_round(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


@pytest.fixture(params=["resident", "pairs", "persistent", "gather"])
def algo(request, env):
    """Runs a test once with each kernel family, for the forward convolution
    (the data gradient is the forward kernel on flipped weights, so it follows
    the choice too) and the weight gradient ("resident": the automatic resident
    choices; "pairs": the resident forward kernel with one block per tile and
    the weight gradient with tap-pair rows only; "persistent": the persistent
    forward kernel wherever its buffers fit)."""
    _, ws, _ = env
    fwd = {"pairs": "pertile"}.get(request.param, request.param)
    wgrad = {"persistent": "resident"}.get(request.param, request.param)
    prev = ws.ws_conv3d_fwd_algo(fwd), ws.ws_conv3d_bwd_weight_algo(wgrad)
    yield request.param
    ws.ws_conv3d_fwd_algo(prev[0])
    ws.ws_conv3d_bwd_weight_algo(prev[1])


@pytest.mark.parametrize("shape,Ci,Co,k", [((2, 6, 5, 7), 32, 48, 3), ((1, 9, 4, 3), 16, 16, 3),
                                           ((1, 8, 8, 8), 96, 64, 3), ((2, 5, 6, 7), 48, 32, 1),
                                           ((1, 8, 8, 12), 64, 224, 3), ((1, 3, 21, 64), 32, 32, 3),
                                           ((2, 3, 13, 64), 16, 96, 3), ((1, 4, 20, 32), 64, 64, 3),
                                           ((1, 4, 9, 12), 96, 32, 3)])
def test_conv_forward_and_gradients(env, algo, shape, Ci, Co, k):
    torch, ws, conv = env
    rng = np.random.default_rng(sum(shape) + Ci + Co + k)
    N, D, H, W = shape
    x = _bf16_round(torch, rng.standard_normal((N, D, H, W, Ci)))
    w = _bf16_round(torch, rng.standard_normal((Co, k, k, k, Ci)) * 0.1)
    b = rng.standard_normal(Co).astype(np.float32)
    dy = _bf16_round(torch, rng.standard_normal((N, D, H, W, Co)))
    dev = torch.device("cuda:0")
    # the input lives in a wider buffer at a channel offset (a concatenation view)
    xbuf = torch.zeros((N, D, H, W, Ci + 16), dtype=torch.bfloat16, device=dev)
    xbuf[..., 16:] = torch.from_numpy(x).to(dev)
    xv = xbuf[..., 16:]
    wt = torch.from_numpy(w).to(dev).to(torch.bfloat16)
    bt = torch.from_numpy(b).to(dev)
    y = torch.zeros((N, D, H, W, Co), dtype=torch.float32, device=dev)
    ws.ws_conv3d_fwd(xv, wt, bt, y, relu=False)
    ref = conv.conv3d_fwd(x, w, b)
    assert _rel(y.cpu().numpy(), ref) < 2e-5
    # ReLU + BF16 output
    yb = torch.zeros((N, D, H, W, Co), dtype=torch.bfloat16, device=dev)
    ws.ws_conv3d_fwd(xv, wt, bt, yb, relu=True)
    assert _rel(yb.float().cpu().numpy(), np.maximum(ref, 0)) < 1e-2
    # data gradient: flipped weights, channels exchanged
    wf = torch.zeros((Ci, k, k, k, Co), dtype=torch.bfloat16, device=dev)
    ws.ws_conv3d_flip_weights(wt, wf)
    dyt = torch.from_numpy(dy).to(dev).to(torch.bfloat16)
    dx = torch.zeros((N, D, H, W, Ci), dtype=torch.float32, device=dev)
    ws.ws_conv3d_fwd(dyt, wf, None, dx, relu=False)
    assert _rel(dx.cpu().numpy(), conv.conv3d_bwd_data(dy, w)) < 2e-5
    # weight and bias gradients (the resident weight-gradient kernel holds 3 Co
    # accumulator columns, so Co > 160 takes the gathered one)
    if algo in ("resident", "pairs", "persistent") and Co > 160:
        ws.ws_conv3d_bwd_weight_algo("auto")
    dw = torch.zeros((Co, k, k, k, Ci), dtype=torch.float32, device=dev)
    db = torch.zeros(Co, dtype=torch.float32, device=dev)
    ws.ws_conv3d_bwd_weight(xv, dyt, dw, db, k)
    rdw, rdb = conv.conv3d_bwd_weight(x, dy, k)
    assert _rel(dw.cpu().numpy(), rdw) < 2e-5
    assert _rel(db.cpu().numpy(), rdb) < 2e-5
    # the chunks are summed in a fixed order: a second call gives the same bits,
    # and the call accumulates into what dw and db hold
    dw2, db2 = torch.zeros_like(dw), torch.zeros_like(db)
    ws.ws_conv3d_bwd_weight(xv, dyt, dw2, db2, k)
    assert torch.equal(dw, dw2) and torch.equal(db, db2)
    ws.ws_conv3d_bwd_weight(xv, dyt, dw2, db2, k)
    assert _rel(dw2.cpu().numpy(), 2 * rdw) < 2e-5 and _rel(db2.cpu().numpy(), 2 * rdb) < 2e-5
    assert ws.ws_tc_status() == 0  # no tensor-core wait gave up


def test_resident_kernel_refuses_wide_lines(env):
    """The resident-tile kernels hold a line plus its two halo columns in one
    TMA box (at most 256 columns): wider lines take the gathered kernels, and
    forcing the resident ones is refused as a bad argument."""
    torch, ws, conv = env
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(5)
    x = _bf16_round(torch, rng.standard_normal((1, 2, 2, 300, 16)))
    w = _bf16_round(torch, rng.standard_normal((16, 3, 3, 3, 16)) * 0.1)
    xt = torch.from_numpy(x).to(dev).to(torch.bfloat16)
    wt = torch.from_numpy(w).to(dev).to(torch.bfloat16)
    y = torch.zeros((1, 2, 2, 300, 16), dtype=torch.float32, device=dev)
    ws.ws_conv3d_fwd(xt, wt, None, y, relu=False)  # automatic: the gathered kernel
    assert _rel(y.cpu().numpy(), conv.conv3d_fwd(x, w)) < 2e-5
    dw = torch.zeros((16, 3, 3, 3, 16), dtype=torch.float32, device=dev)
    ws.ws_conv3d_bwd_weight(xt, xt, dw, None, 3)  # automatic: the gathered kernel
    assert _rel(dw.cpu().numpy(), conv.conv3d_bwd_weight(x, x, 3)[0]) < 2e-5
    prev = ws.ws_conv3d_fwd_algo("resident"), ws.ws_conv3d_bwd_weight_algo("resident")
    try:
        with pytest.raises(ws.WsError):
            ws.ws_conv3d_fwd(xt, wt, None, y, relu=False)
        with pytest.raises(ws.WsError):
            ws.ws_conv3d_bwd_weight(xt, xt, dw, None, 3)
    finally:
        ws.ws_conv3d_fwd_algo(prev[0])
        ws.ws_conv3d_bwd_weight_algo(prev[1])
    assert ws._lib().ws_conv3d_fwd_algo(5) == -1 and ws._lib().ws_conv3d_bwd_weight_algo(4) == -1
    assert ws.ws_tc_status() == 0


def test_pool_upsample_relu(env):
    torch, ws, _ = env
    rng = np.random.default_rng(7)
    dev = torch.device("cuda:0")
    x = _bf16_round(torch, rng.standard_normal((2, 4, 6, 8, 16)))
    xt = torch.from_numpy(x).to(dev).to(torch.bfloat16)
    y = torch.zeros((2, 2, 3, 4, 16), dtype=torch.bfloat16, device=dev)
    ws.ws_avgpool2(xt, y)
    ref = x.reshape(2, 2, 2, 3, 2, 4, 2, 16).mean(axis=(2, 4, 6))
    assert _rel(y.float().cpu().numpy(), ref) < 1e-2
    up = torch.zeros((2, 4, 6, 8, 16), dtype=torch.bfloat16, device=dev)
    ws.ws_upsample2(y, up)
    u = y.float().cpu().numpy()
    assert np.array_equal(up.float().cpu().numpy(), u.repeat(2, 1).repeat(2, 2).repeat(2, 3))
    # adjoints: <pool(x), g> = <x, pool_bwd(g)>, <up(z), h> = <z, up_bwd(h)>
    g = torch.from_numpy(_bf16_round(torch, rng.standard_normal((2, 2, 3, 4, 16)))).to(dev).to(torch.bfloat16)
    dx = torch.zeros_like(xt)
    ws.ws_avgpool2_bwd(g, dx)
    assert np.allclose(dx.float().cpu().numpy(), g.float().cpu().numpy().repeat(2, 1).repeat(2, 2).repeat(2, 3) / 8)
    h = torch.from_numpy(_bf16_round(torch, rng.standard_normal((2, 4, 6, 8, 16)))).to(dev).to(torch.bfloat16)
    dz = torch.zeros_like(y)
    ws.ws_upsample2_bwd(h, dz)
    hs = h.float().cpu().numpy().reshape(2, 2, 2, 3, 2, 4, 2, 16).sum(axis=(2, 4, 6))
    assert _rel(dz.float().cpu().numpy(), hs) < 1e-2
    # ReLU adjoint
    dy = torch.ones_like(xt)
    ws.ws_relu_bwd(xt, dy)
    assert np.array_equal(dy.float().cpu().numpy(), (x > 0).astype(np.float32))


def test_mse_and_adam(env):
    torch, ws, _ = env
    rng = np.random.default_rng(8)
    dev = torch.device("cuda:0")
    P, C = 1000, 5
    pred = rng.standard_normal((P, 16)).astype(np.float32)
    tgt = rng.standard_normal((P, C)).astype(np.float32)
    mask = (rng.random(P) < 0.7).astype(np.uint8)
    wch = np.array([1, 2, 3, 4, 5], np.float32)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    dpred = torch.zeros((P, 16), dtype=torch.bfloat16, device=dev)
    ws.ws_mse_loss(torch.from_numpy(pred).to(dev), torch.from_numpy(tgt).to(dev), torch.from_numpy(mask).to(dev),
                   torch.from_numpy(wch).to(dev), dpred, loss)
    d = (pred[:, :C] - tgt) * mask[:, None]
    ref_loss = float((wch * d * d).sum() / (P * C))
    assert abs(float(loss.item()) - ref_loss) < 1e-5 * ref_loss
    ref_g = np.zeros((P, 16), np.float32)
    ref_g[:, :C] = 2 * wch * d / (P * C)
    assert _rel(dpred.float().cpu().numpy(), ref_g) < 1e-2
    # one Adam step
    n = 777
    w = rng.standard_normal(n).astype(np.float32)
    g = rng.standard_normal(n).astype(np.float32)
    wt, m, v = (torch.from_numpy(w.copy()).to(dev), torch.zeros(n, device=dev), torch.zeros(n, device=dev))
    wb = torch.zeros(n, dtype=torch.bfloat16, device=dev)
    ws.ws_adam(wt, m, v, torch.from_numpy(g).to(dev), wb, lr_t=1e-3)
    mr = 0.1 * g
    vr = 0.001 * g * g
    wr = w - 1e-3 * mr / (np.sqrt(vr) + 1e-8)
    assert np.allclose(wt.cpu().numpy(), wr, rtol=1e-5, atol=1e-7)
    assert np.allclose(wb.float().cpu().numpy(), wr, rtol=1e-2, atol=1e-3)
