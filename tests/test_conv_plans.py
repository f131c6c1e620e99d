"""Host-side tiling of the resident-tile convolution kernels (no GPU needed).

ws_conv3d_plan returns the plan the library would launch for a shape.  These
tests check, for a grid of shapes, that every plan stays inside the hardware
limits the kernels rely on (tensor-memory columns, shared memory per block and
per SM, TMA box extents, mbarrier transaction counts, the rows each shifted
descriptor reaches).  They also replay each kernel's tiling in NumPy, using the
returned plan: the loads of the TMA boxes (zeros outside the volume), the
shifted descriptor views and the accumulation per tile or K-block.  The replay
must give the direct 3x3x3 correlation, so a wrong shift, halo or row mapping
in the plan's arithmetic shows up on the CPU.
"""
import itertools
import math

import numpy as np
import pytest

SMEM_PER_SM, SMEM_PER_BLOCK, SMEM_RESERVED = 233472, 232448, 1024


@pytest.fixture(scope="module")
def ws():
    from paper_1711_03254_gb300 import ws as w
    return w


@pytest.fixture
def algos(ws):
    """Restores the process-wide kernel choices after a test."""
    prev = ws.ws_conv3d_fwd_algo("auto"), ws.ws_conv3d_bwd_weight_algo("auto")
    yield
    ws.ws_conv3d_fwd_algo(prev[0])
    ws.ws_conv3d_bwd_weight_algo(prev[1])


def _resident_per_sm(smem):
    return SMEM_PER_SM // (smem + SMEM_RESERVED)


SHAPES = [(N, D, H, W) for N, D in ((1, 1), (2, 5)) for H in (1, 5, 13, 64) for W in (1, 3, 7, 12, 16, 32, 64, 200, 254)]


@pytest.mark.parametrize("fwd_algo", ["resident", "pertile", "persistent"])
def test_forward_plans_stay_within_limits(ws, algos, fwd_algo):
    ws.ws_conv3d_fwd_algo(fwd_algo)
    n = 0
    for (N, D, H, W), Ci, Co in itertools.product(SHAPES, (16, 32, 96), (16, 32, 64, 96, 224)):
        p = ws.ws_conv3d_plan("fwd", N, D, H, W, Ci, Co)
        assert p is not None, (N, D, H, W, Ci, Co)
        n += 1
        pitch, by = p["pitch"], p["by"]
        assert pitch == W + 2 <= 256 and 1 <= by <= H and by + 2 <= 256
        assert p["nyt"] == math.ceil(H / by)
        assert p["ntiles"] == math.ceil(((by - 1) * pitch + W) / 128)
        rows = p["a_half"] // 16
        # the TMA box and every row a tap's descriptor reaches lie in one K half
        assert (by + 2) * pitch <= rows and 128 * p["ntiles"] - 1 + 2 * pitch + 2 < rows
        assert p["stage_bytes"] == 2 * p["a_half"] + 18 * Co * 16 and p["a_half"] % 128 == 0
        assert p["tx_bytes"] == 2 * (by + 2) * pitch * 16 + 18 * Co * 16 < 1 << 20
        assert p["stages"] >= 2 and p["smem"] <= SMEM_PER_BLOCK
        barriers = 2 * p["stages"] + (5 if p["persistent"] else 1)
        assert 1023 + p["stages"] * p["stage_bytes"] + 8 * barriers + 8 <= p["smem"]
        assert p["stages"] * p["stage_bytes"] + 1024 <= 256 * 1024  # 14-bit descriptor address field
        cols = p["cols"]
        assert cols in (32, 64, 128, 256, 512)
        if p["persistent"]:
            assert fwd_algo != "pertile" and (fwd_algo == "persistent" or Co >= 64 or Ci <= 16)
            assert p["buf_cols"] >= p["ntiles"] * Co and cols == 2 * p["buf_cols"] <= 512
            assert _resident_per_sm(p["smem"]) == 1
        else:
            assert p["buf_cols"] == 0 and p["ntiles"] * Co <= cols
            assert _resident_per_sm(p["smem"]) * cols <= 512  # tensor memory of the resident blocks
            assert p["grid"] == N * D * p["nyt"]
    assert n == len(SHAPES) * 15
    # lines wider than a TMA box take the gathered kernel
    assert ws.ws_conv3d_plan("fwd", 1, 2, 2, 255, 16, 16) is None


@pytest.mark.parametrize("wg_algo", ["resident", "pairs"])
def test_weight_gradient_plans_stay_within_limits(ws, algos, wg_algo):
    ws.ws_conv3d_bwd_weight_algo(wg_algo)
    planned = 0
    for (N, D, H, W), Ci, Co in itertools.product(SHAPES, (16, 32, 64, 96, 128), (16, 32, 48, 64, 160)):
        p = ws.ws_conv3d_plan("wgrad", N, D, H, W, Ci, Co)
        if p is None:
            # only where not even two stages of one-line K-blocks fit (the gathered kernel runs)
            rows1 = (math.ceil((W + 2) / 16) * 16 + 2 + 7) // 8 * 8
            assert 2 * (16 + Co // 8) * rows1 * 16 + 1024 + 56 > SMEM_PER_BLOCK, (N, D, H, W, Ci, Co)
            continue
        planned += 1
        pitch, by, rows = p["pitch"], p["by"], p["region"] // 16
        assert pitch == W + 2 <= 256 and 1 <= by <= H and p["nyb"] == math.ceil(H / by)
        assert p["ksteps"] == math.ceil(by * pitch / 16)
        nkb = N * D * p["nyb"]
        assert p["npb"] * p["kpb"] >= nkb > (p["npb"] - 1) * p["kpb"]
        assert p["stages"] >= 2 and p["smem"] <= SMEM_PER_BLOCK and p["region"] % 128 == 0
        assert 1023 + p["stages"] * p["stage_bytes"] + 8 * (2 * p["stages"] + 1) + 8 <= p["smem"]
        assert _resident_per_sm(p["smem"]) * p["cols"] <= 512
        if p["dz"]:
            assert wg_algo == "resident" and Ci % 32 == 0 and Co <= 48
            assert p["ci_blk"] == 32 and 9 * Co <= p["cols"] and p["grid_y"] == Ci // 32
            assert rows >= (by + 2) * pitch and rows > p["ksteps"] * 16 + 2 * pitch + 1
            assert p["stage_bytes"] == max(16, 13 + Co // 8) * p["region"]
            assert (12 * (by + 2) * pitch + Co // 8 * by * pitch) * 16 < 1 << 20
        else:
            assert p["J"] * p["ci_blk"] == 128 and Ci % p["ci_blk"] == 0
            assert p["ntile"] == math.ceil(9 / p["J"]) and 3 * Co <= p["cols"]
            assert rows >= by * pitch and rows > p["ksteps"] * 16 + 1
            assert p["stage_bytes"] == (16 + Co // 8) * p["region"]
            assert (16 + Co // 8) * by * pitch * 16 < 1 << 20
    assert planned > 0.9 * len(SHAPES) * 25
    # more than 160 output channels: the gathered kernel (3 Co accumulator columns)
    assert ws.ws_conv3d_plan("wgrad", 1, 2, 4, 8, 32, 176) is None


# ---------------------------------------------------------------- replays of the tiling
def _direct(x, w):
    """y[n,z,y,x,co] = sum_t,ci w[co,t,ci] x[p + t - 1, ci] with zero padding; w [Co, 27, Ci]."""
    N, D, H, W, Ci = x.shape
    xp = np.zeros((N, D + 2, H + 2, W + 2, Ci))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    y = np.zeros((N, D, H, W, w.shape[0]))
    for t in range(27):
        tz, ty, tx = t // 9, (t // 3) % 3, t % 3
        y += xp[:, tz:tz + D, ty:ty + H, tx:tx + W] @ w[:, t].T
    return y


def _direct_wgrad(x, dy):
    """dW[co, t, ci] = sum_p dy[p, co] x[p + t - 1, ci]."""
    N, D, H, W, Ci = x.shape
    Co = dy.shape[-1]
    xp = np.zeros((N, D + 2, H + 2, W + 2, Ci))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    dw = np.zeros((Co, 27, Ci))
    for t in range(27):
        tz, ty, tx = t // 9, (t // 3) % 3, t % 3
        dw[:, t] = dy.reshape(-1, Co).T @ xp[:, tz:tz + D, ty:ty + H, tx:tx + W].reshape(-1, Ci)
    return dw


def _box(t, c0, x0, y0, z, n, pitch, lines):
    """A TMA box of 8 channels: rows (line, column) from (x0, y0) of plane z, zeros outside."""
    N, D, H, W, C = t.shape
    out = np.zeros((lines, pitch, 8))
    if 0 <= z < D:
        ys, xs = y0 + np.arange(lines), x0 + np.arange(pitch)
        vy, vx = (ys >= 0) & (ys < H), (xs >= 0) & (xs < W)
        out[np.ix_(vy, vx)] = t[n, z][np.ix_(ys[vy], xs[vx])][..., c0:c0 + 8]
    return out.reshape(lines * pitch, 8)


def _replay_forward(x, w, p, shift=0):
    """The resident forward tiling: per tile and K-step (16-channel chunk c, plane dz) the two
    K halves of the padded plane slice, and for each M tile j and tap (dy, dx) the 128 rows
    from row 128 j + dy (W + 2) + dx of that slice."""
    N, D, H, W, Ci = x.shape
    Co = w.shape[0]
    pitch, by, rows = p["pitch"], p["by"], p["a_half"] // 16
    y = np.full((N, D, H, W, Co), np.nan)
    for tile in range(N * D * p["nyt"]):
        yt, zn = tile % p["nyt"], tile // p["nyt"]
        z, n = zn % D, zn // D
        y0 = yt * by
        lt = min(by, H - y0)
        nt = math.ceil(((lt - 1) * pitch + W) / 128)
        acc = np.zeros((nt * 128, Co))
        for c in range(Ci // 16):
            for dz in range(3):
                if not 0 <= z + dz - 1 < D:
                    continue  # the kernel skips K-steps outside the volume
                a = np.zeros((rows, 16))
                for h in range(2):
                    a[:(by + 2) * pitch, 8 * h:8 * h + 8] = _box(x, 16 * c + 8 * h, -1, y0 - 1, z + dz - 1, n, pitch, by + 2)
                for j in range(nt):
                    for t9 in range(9):
                        r0 = 128 * j + (t9 // 3) * pitch + t9 % 3 + shift
                        assert r0 + 128 <= rows
                        acc[128 * j:128 * j + 128] += a[r0:r0 + 128] @ w[:, dz * 9 + t9, 16 * c:16 * c + 16].T
        q = np.arange(nt * 128)
        line, col = q // pitch, q % pitch
        ok = (col < W) & (line < lt)
        y[n, z, y0 + line[ok], col[ok]] = acc[ok]
    return y


@pytest.mark.parametrize("fwd_algo", ["resident", "pertile", "persistent"])
@pytest.mark.parametrize("shape,Ci,Co", [((1, 3, 9, 12), 32, 32), ((2, 2, 5, 7), 16, 48), ((1, 2, 7, 40), 32, 64),
                                         ((1, 3, 4, 3), 16, 16)])
def test_forward_tiling_replays_the_correlation(ws, algos, fwd_algo, shape, Ci, Co):
    ws.ws_conv3d_fwd_algo(fwd_algo)
    rng = np.random.default_rng(sum(shape) + Ci + Co)
    x = rng.standard_normal(shape + (Ci,))
    w = rng.standard_normal((Co, 27, Ci))
    p = ws.ws_conv3d_plan("fwd", *shape, Ci, Co)
    y = _replay_forward(x, w, p)
    ref = _direct(x, w)
    assert not np.isnan(y).any()  # every output written by exactly the rows the epilogue keeps
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()


def test_forward_replay_catches_a_wrong_tap_offset(ws, algos):
    """A descriptor one row off (the tap offset dy (W + 2) + dx + 1) must not pass."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1, 2, 5, 7, 16))
    w = rng.standard_normal((16, 27, 16))
    p = ws.ws_conv3d_plan("fwd", 1, 2, 5, 7, 16, 16)
    y = _replay_forward(x, w, p, shift=1)
    assert np.abs(y - _direct(x, w)).max() > 1e-3


def _replay_wgrad(x, dy, p):
    """The resident weight-gradient tiling.  Per block (position block pb, channel block cb,
    tile) and K-block (by lines of a plane): the X boxes of its slots, the dY box (columns
    0 .. W + 1, zeros past W), then per K-step of 16 rows the MN-major A (16 regions of 8
    channels) against B, A shifted by dx rows (tap pairs) or by dy (W + 2) + dx rows (dz
    slots).  Unused slots hold zeros, and the first free slot of channel block 0 holds ones:
    its first row is the bias gradient.  Returns (dW [Co, 27, Ci], db [Co])."""
    N, D, H, W, Ci = x.shape
    Co = dy.shape[-1]
    pitch, by, rows = p["pitch"], p["by"], p["region"] // 16
    G, NB, cb_n = p["ci_blk"] // 8, Co // 8, Ci // p["ci_blk"]
    nkb = N * D * p["nyb"]
    dw = np.zeros((Co, 27, Ci))
    db = np.zeros(Co)
    for pb, cb, ti in itertools.product(range(p["npb"]), range(cb_n), range(p["ntile"])):
        kbs = range(pb * p["kpb"], min((pb + 1) * p["kpb"], nkb))
        if p["dz"]:
            slots = [(dz, None) for dz in range(3)]  # slot 3: ones (channel block 0) or unused
            ones_slot = 3 if cb == 0 else None
            shifts = [(dyy * pitch + dx, dyy * 3 + dx) for dyy in range(3) for dx in range(3)]
        else:
            J = p["J"]
            slots = [((ti * J + j) // 3, (ti * J + j) % 3) for j in range(J) if ti * J + j < 9]
            ones_slot = len(slots) if cb == 0 and ti == p["ntile"] - 1 and len(slots) < J else None
            shifts = [(dx, dx) for dx in range(3)]
        nslot = 128 // p["ci_blk"]
        a = np.zeros((rows, 128))
        if ones_slot is not None:
            a[:, ones_slot * p["ci_blk"]:ones_slot * p["ci_blk"] + 8] = 1.0
        b = np.zeros((rows, Co))
        acc = np.zeros((len(shifts), 128, Co))
        for kb in kbs:
            yb, z, n = kb % p["nyb"], (kb // p["nyb"]) % D, kb // (p["nyb"] * D)
            y0 = yb * by
            for s, (dz, dyy) in enumerate(slots):
                lines, ly0 = (by + 2, y0 - 1) if p["dz"] else (by, y0 + dyy - 1)
                for g in range(G):
                    col = s * p["ci_blk"] + 8 * g
                    a[:lines * pitch, col:col + 8] = _box(x, cb * p["ci_blk"] + 8 * g, -1, ly0, z + dz - 1, n, pitch, lines)
            for g in range(NB):
                b[:by * pitch, 8 * g:8 * g + 8] = _box(dy, 8 * g, 0, y0, z, n, pitch, by)
            for ks in range(p["ksteps"]):
                for k, (off, _) in enumerate(shifts):
                    r0 = 16 * ks + off
                    assert r0 + 16 <= rows
                    acc[k] += a[r0:r0 + 16].T @ b[16 * ks:16 * ks + 16]
        for k, (_, tap_in_slot) in enumerate(shifts):
            for s, (dz, dyy) in enumerate(slots):
                t = dz * 9 + tap_in_slot if p["dz"] else (dz * 3 + dyy) * 3 + tap_in_slot
                ci = slice(cb * p["ci_blk"], (cb + 1) * p["ci_blk"])
                dw[:, t, ci] += acc[k, s * p["ci_blk"]:(s + 1) * p["ci_blk"]].T
        if ones_slot is not None:
            db += acc[0, ones_slot * p["ci_blk"]]
        assert nslot * p["ci_blk"] == 128
    return dw, db


@pytest.mark.parametrize("wg_algo", ["resident", "pairs"])
@pytest.mark.parametrize("shape,Ci,Co", [((1, 3, 6, 12), 32, 32), ((2, 2, 5, 9), 64, 64), ((1, 2, 4, 7), 16, 16),
                                         ((1, 2, 3, 10), 96, 48), ((1, 2, 3, 5), 128, 16)])
def test_weight_gradient_tiling_replays_the_correlation(ws, algos, wg_algo, shape, Ci, Co):
    ws.ws_conv3d_bwd_weight_algo(wg_algo)
    rng = np.random.default_rng(sum(shape) + Ci + Co)
    x = rng.standard_normal(shape + (Ci,))
    dy = rng.standard_normal(shape + (Co,))
    p = ws.ws_conv3d_plan("wgrad", *shape, Ci, Co)
    assert p["dz"] == (wg_algo == "resident" and Ci % 32 == 0 and Co <= 48)
    dw, db = _replay_wgrad(x, dy, p)
    ref = _direct_wgrad(x, dy)
    assert np.abs(dw - ref).max() <= 1e-12 * np.abs(ref).max()
    if p["dz"] or p["J"] * p["ntile"] > 9:  # the bias rides in a free slot
        ref_b = dy.reshape(-1, Co).sum(axis=0)
        assert np.abs(db - ref_b).max() <= 1e-12 * np.abs(ref_b).max()
