"""Python binding of include/ws.h (argument marshalling only).

Each function takes torch CUDA tensors (device memory owned by the caller)
and calls the kernel of the same name in liblbm_gb300.so.  Activations are
channels-last BF16 tensors shaped [N, D, H, W, ld]; a channel slice
``t[..., c0:c1]`` can be passed as a view (row stride ld, offset c0).
"""
from __future__ import annotations

import ctypes

from . import lbm as _lbm

_sig_done = False


def _lib():
    global _sig_done
    L = _lbm.library()
    if not _sig_done:
        vp, i, ll, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_float
        L.ws_conv3d_fwd.argtypes = [vp, i, vp, vp, vp, i, i, i, i, i, i, i, i, i, i, vp]
        L.ws_conv3d_fwd_algo.argtypes = [i]
        L.ws_conv3d_bwd_weight_algo.argtypes = [i]
        L.ws_conv3d_plan.argtypes = [i, i, i, i, i, i, i, ctypes.POINTER(ll), i]
        L.ws_conv3d_flip_weights.argtypes = [vp, vp, i, i, i, vp]
        L.ws_conv3d_bwd_weight.argtypes = [vp, i, vp, i, vp, vp, i, i, i, i, i, i, i, vp]
        L.ws_avgpool2.argtypes = [vp, i, vp, i, i, i, i, i, i, vp]
        L.ws_avgpool2_bwd.argtypes = [vp, i, vp, i, i, i, i, i, i, i, vp]
        L.ws_upsample2.argtypes = [vp, i, vp, i, i, i, i, i, i, vp]
        L.ws_upsample2_bwd.argtypes = [vp, i, vp, i, i, i, i, i, i, i, vp]
        L.ws_relu_bwd.argtypes = [vp, i, vp, i, ll, i, vp]
        L.ws_mse_loss.argtypes = [vp, i, vp, vp, vp, vp, i, vp, ll, i, vp]
        L.ws_adam.argtypes = [vp, vp, vp, vp, vp, ll, f, f, f, f, f, vp]
        L.ws_to_bf16.argtypes = [vp, i, vp, i, ll, i, vp]
        L.ws_tc_status.argtypes = [vp]
        for name in ("ws_conv3d_fwd", "ws_conv3d_fwd_algo", "ws_conv3d_flip_weights", "ws_conv3d_bwd_weight",
                     "ws_conv3d_bwd_weight_algo", "ws_avgpool2", "ws_avgpool2_bwd", "ws_upsample2",
                     "ws_upsample2_bwd", "ws_relu_bwd", "ws_mse_loss", "ws_adam",
                     "ws_to_bf16", "ws_tc_status", "ws_conv3d_plan"):
            getattr(L, name).restype = ctypes.c_int
        _sig_done = True
    return L


class WsError(RuntimeError):
    pass


def _ok(rc, name):
    if rc != 0:
        raise WsError(f"{name} returned {rc}")


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _ld(t):
    """Row stride (elements) of a channels-last view."""
    return t.stride(-2) if t.dim() >= 2 else t.shape[-1]


def _vol(t):
    N, D, H, W = t.shape[:4]
    return N, D, H, W


def ws_conv3d_fwd(x, w, bias, y, relu: bool):
    """x: bf16 [N,D,H,W,Ci] view; w: bf16 [Co,k,k,k,Ci]; y: bf16 or fp32 [N,D,H,W,Co] view."""
    import torch
    N, D, H, W = _vol(x)
    Co, k, Ci = w.shape[0], w.shape[1], w.shape[4]
    rc = _lib().ws_conv3d_fwd(x.data_ptr(), _ld(x), w.data_ptr(), bias.data_ptr() if bias is not None else None,
                              y.data_ptr(), _ld(y), int(y.dtype == torch.float32), N, D, H, W, Ci, Co, k, int(relu),
                              _stream())
    _ok(rc, "ws_conv3d_fwd")


def ws_conv3d_fwd_algo(algo: str) -> str:
    """Forward kernel of later ws_conv3d_fwd calls: "auto", "gather",
    "resident", "pertile" (resident, one block per tile, never persistent) or
    "persistent" (resident, persistent wherever its buffers fit); returns the
    previous choice."""
    names = ("auto", "gather", "resident", "pertile", "persistent")
    prev = _lib().ws_conv3d_fwd_algo(names.index(algo))
    if prev < 0:
        raise WsError(f"ws_conv3d_fwd_algo rejected {algo}")
    return names[prev]


def ws_conv3d_bwd_weight_algo(algo: str) -> str:
    """Weight-gradient kernel of later ws_conv3d_bwd_weight calls: "auto",
    "gather", "resident" or "pairs" (resident, tap-pair rows only); returns
    the previous choice."""
    names = ("auto", "gather", "resident", "pairs")
    prev = _lib().ws_conv3d_bwd_weight_algo(names.index(algo))
    if prev < 0:
        raise WsError(f"ws_conv3d_bwd_weight_algo rejected {algo}")
    return names[prev]


_FWD_PLAN = ("persistent", "by", "nyt", "pitch", "ntiles", "stages", "cols", "per_sm", "a_half", "stage_bytes",
             "tx_bytes", "smem", "grid", "buf_cols")
_WGRAD_PLAN = ("dz", "by", "nyb", "pitch", "ksteps", "J", "ci_blk", "ntile", "npb", "kpb", "stages", "cols",
               "region", "stage_bytes", "smem", "grid_y")


def ws_conv3d_plan(which: str, N: int, D: int, H: int, W: int, Ci: int, Co: int):
    """Tiling of the resident-tile kernels for a 3x3x3 convolution ("fwd" or
    "wgrad") under the current kernel choice, as a dict; None where the
    gathered kernel would run.  Host only."""
    names = _FWD_PLAN if which == "fwd" else _WGRAD_PLAN
    out = (ctypes.c_longlong * 16)()
    n = _lib().ws_conv3d_plan(0 if which == "fwd" else 1, N, D, H, W, Ci, Co, out, 16)
    if n == -1:
        return None
    if n < 0:
        raise WsError(f"ws_conv3d_plan rejected {which} {(N, D, H, W, Ci, Co)}")
    return dict(zip(names, out[:n]))


def ws_conv3d_flip_weights(w, wf):
    Co, k, Ci = w.shape[0], w.shape[1], w.shape[4]
    _ok(_lib().ws_conv3d_flip_weights(w.data_ptr(), wf.data_ptr(), Co, Ci, k, _stream()), "ws_conv3d_flip_weights")


def ws_conv3d_bwd_weight(x, dy, dw, db, k: int):
    N, D, H, W = _vol(x)
    Ci, Co = x.shape[-1], dy.shape[-1]
    rc = _lib().ws_conv3d_bwd_weight(x.data_ptr(), _ld(x), dy.data_ptr(), _ld(dy), dw.data_ptr(),
                                     db.data_ptr() if db is not None else None, N, D, H, W, Ci, Co, k, _stream())
    _ok(rc, "ws_conv3d_bwd_weight")


def ws_avgpool2(x, y):
    N, D, H, W = _vol(x)
    _ok(_lib().ws_avgpool2(x.data_ptr(), _ld(x), y.data_ptr(), _ld(y), N, D, H, W, x.shape[-1], _stream()),
        "ws_avgpool2")


def ws_avgpool2_bwd(dy, dx, accumulate: bool = False):
    N, D, H, W = _vol(dx)
    _ok(_lib().ws_avgpool2_bwd(dy.data_ptr(), _ld(dy), dx.data_ptr(), _ld(dx), N, D, H, W, dx.shape[-1],
                               int(accumulate), _stream()), "ws_avgpool2_bwd")


def ws_upsample2(x, y):
    N, D, H, W = _vol(x)
    _ok(_lib().ws_upsample2(x.data_ptr(), _ld(x), y.data_ptr(), _ld(y), N, D, H, W, x.shape[-1], _stream()),
        "ws_upsample2")


def ws_upsample2_bwd(dy, dx, accumulate: bool = False):
    N, D, H, W = _vol(dx)
    _ok(_lib().ws_upsample2_bwd(dy.data_ptr(), _ld(dy), dx.data_ptr(), _ld(dx), N, D, H, W, dx.shape[-1],
                                int(accumulate), _stream()), "ws_upsample2_bwd")


def ws_relu_bwd(y, dy):
    P = y.numel() // y.shape[-1]
    _ok(_lib().ws_relu_bwd(y.data_ptr(), _ld(y), dy.data_ptr(), _ld(dy), P, y.shape[-1], _stream()), "ws_relu_bwd")


def ws_mse_loss(pred, target, mask, wch, dpred, loss):
    C = target.shape[-1]
    P = target.numel() // C
    _ok(_lib().ws_mse_loss(pred.data_ptr(), _ld(pred), target.data_ptr(), mask.data_ptr(), wch.data_ptr(),
                           dpred.data_ptr(), _ld(dpred), loss.data_ptr(), P, C, _stream()), "ws_mse_loss")


def ws_adam(w, m, v, g, wb, lr_t, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
    _ok(_lib().ws_adam(w.data_ptr(), m.data_ptr(), v.data_ptr(), g.data_ptr(), wb.data_ptr() if wb is not None else None,
                       w.numel(), float(lr_t), float(beta1), float(beta2), float(eps), float(weight_decay), _stream()),
        "ws_adam")


def ws_to_bf16(x, y):
    C = y.shape[-1]
    P = y.numel() // C if y.is_contiguous() else x.numel() // x.shape[-1]
    _ok(_lib().ws_to_bf16(x.data_ptr(), _ld(x), y.data_ptr(), _ld(y), P, C, _stream()), "ws_to_bf16")


def ws_tc_status() -> int:
    """0 when no tensor-core convolution since the last call gave up on a
    bounded wait, 5 otherwise (waits for the current stream; clears the record)."""
    return int(_lib().ws_tc_status(_stream()))
