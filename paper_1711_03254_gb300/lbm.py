"""Python binding of the C ABI in include/lbm.h (argument marshalling only).

Every function here has the name of the C entry point it calls; all
computation happens in the CUDA library ``liblbm_gb300.so``.  There is no CPU
fallback: importing this module without the built library raises.

Arrays are NumPy, C order: cell types uint8 [batch, nz, ny, nx], densities
float64 [batch, nz, ny, nx], velocity float64 [batch, nz, ny, nx, 3].
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm_gb300.so")

LBM_FP64, LBM_FP32, LBM_FP32_F16S, LBM_FP32_BF16S = 0, 1, 2, 3
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16s": LBM_FP32_F16S, "bf16s": LBM_FP32_BF16S}
LBM_KERNEL_AUTO, LBM_KERNEL_TWO_PASS, LBM_KERNEL_FUSED, LBM_KERNEL_CLUSTER = 0, 1, 2, 3
KERNELS = {"auto": 0, "two_pass": 1, "fused": 2, "cluster": 3, "compact": 4, "fused_compact": 5, "persistent": 6}
STATUS = {0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_CUDA", 3: "LBM_ERR_OOM", 4: "LBM_ERR_DIVERGED",
          5: "LBM_ERR_TIMEOUT", 6: "LBM_ERR_STATE"}


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class lbm_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("batch", ctypes.c_int),
                ("precision", ctypes.c_int), ("eq_order", ctypes.c_int), ("wall_model", ctypes.c_int),
                ("reg_order", ctypes.c_int)]


class lbm_instance_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double * 2), ("G", ctypes.c_double), ("rho_s", ctypes.c_double),
                ("g", ctypes.c_double * 3), ("rho_in", ctypes.c_double * 2), ("u_in", ctypes.c_double * 3),
                ("slip", ctypes.c_double)]


_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_lib = None
_hooks = []  # installed allocator hooks (kept alive, see lbm_set_allocator)


def library() -> ctypes.CDLL:
    """Load liblbm_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1711_03254_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
        L.lbm_create.argtypes = [ctypes.POINTER(lbm_config), ctypes.POINTER(lbm_instance_params),
                                 ctypes.POINTER(vp)]
        L.lbm_set_geometry.argtypes = [vp, ctypes.POINTER(ctypes.c_uint8)]
        L.lbm_set_fields.argtypes = [vp, dp, dp, dp]
        L.lbm_step.argtypes = [vp, ctypes.c_int]
        L.lbm_get_fields.argtypes = [vp, dp, dp, dp]
        L.lbm_reduce.argtypes = [vp, dp]
        L.lbm_get_distributions.argtypes = [vp, dp]
        L.lbm_set_distributions.argtypes = [vp, dp]
        L.lbm_get_state.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
        L.lbm_set_state.argtypes = [vp, vp, ctypes.c_size_t]
        L.lbm_set_stream.argtypes = [vp, vp]
        L.lbm_set_kernel.argtypes = [vp, ctypes.c_int]
        L.lbm_set_tiling.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.lbm_autotune.argtypes = [vp, ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]
        L.lbm_run_to_steady.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), dp]
        L.lbm_launch_count.argtypes = [vp]
        L.lbm_launch_count.restype = ctypes.c_longlong
        L.lbm_set_allocator.argtypes = [_ALLOC_T, _FREE_T]
        L.lbm_last_error.argtypes = [vp]
        L.lbm_last_error.restype = ctypes.c_char_p
        L.lbm_destroy.argtypes = [vp]
        L.lbm_destroy.restype = None
        L.lbm_step_part.argtypes = [vp, ctypes.c_int]
        L.lbm_set_params.argtypes = [vp, ctypes.POINTER(lbm_instance_params)]
        L.lbm_plane_bytes.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
        L.lbm_plane_copy.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int]
        L.lbm_set_barrier_test.argtypes = [vp, ctypes.c_longlong, ctypes.c_uint]
        for name in ("lbm_create", "lbm_set_geometry", "lbm_set_fields", "lbm_step", "lbm_get_fields",
                     "lbm_reduce", "lbm_get_distributions", "lbm_set_distributions", "lbm_get_state", "lbm_set_state", "lbm_set_stream", "lbm_set_kernel", "lbm_set_tiling", "lbm_autotune", "lbm_run_to_steady",
                     "lbm_set_allocator", "lbm_step_part", "lbm_plane_bytes", "lbm_plane_copy", "lbm_set_params",
                     "lbm_set_barrier_test"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int, ctx=None, allow=()):
    if rc != 0 and rc not in allow:
        msg = library().lbm_last_error(ctx).decode()
        raise LbmError(rc, msg)
    return rc


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def lbm_set_allocator(alloc=None, release=None):
    """Install a device allocator (python callables alloc(bytes, stream) -> int,
    release(ptr, stream)); with no arguments restore cudaMalloc."""
    if alloc is None:
        return _check(library().lbm_set_allocator(_ALLOC_T(), _FREE_T()))
    a = _ALLOC_T(lambda n, s: alloc(n, s))
    f = _FREE_T(lambda p, s: release(p, s))
    # contexts created while a hook is installed keep calling it until they are
    # destroyed, so every hook stays alive for the life of the process
    _hooks.append((a, f))
    return _check(library().lbm_set_allocator(a, f))


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    import torch

    def alloc(n, stream):
        return int(torch.cuda.caching_allocator_alloc(int(n), torch.cuda.current_device(), stream))

    def release(p, stream):
        torch.cuda.caching_allocator_delete(int(p))

    lbm_set_allocator(alloc, release)


def make_config(nx, ny, nz, batch=1, precision="fp64", eq_order=0, wall_model=2, reg_order=2):
    c = lbm_config()
    c.nx, c.ny, c.nz, c.batch = int(nx), int(ny), int(nz), int(batch)
    c.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    c.eq_order, c.wall_model, c.reg_order = int(eq_order), int(wall_model), int(reg_order)
    return c


def make_params(params):
    arr = (lbm_instance_params * len(params))()
    for k, p in enumerate(params):
        arr[k].tau[:] = [float(v) for v in p.get("tau", (1.0, 1.0))]
        arr[k].G = float(p.get("G", 0.0))
        arr[k].rho_s = float(p.get("rho_s", 0.0))
        arr[k].g[:] = [float(v) for v in p.get("g", (0.0, 0.0, 0.0))]
        arr[k].rho_in[:] = [float(v) for v in p.get("rho_in", (0.0, 0.0))]
        arr[k].u_in[:] = [float(v) for v in p.get("u_in", (0.0, 0.0, 0.0))]
        arr[k].slip = float(p.get("slip", 0.0))
    return arr


def lbm_create(cfg: lbm_config, params) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(library().lbm_create(ctypes.byref(cfg), params, ctypes.byref(h)))
    return h


def lbm_set_params(ctx, params):
    """Replace the per-instance parameters (list of dicts as for Sim) between updates."""
    arr = make_params(params)
    return _check(library().lbm_set_params(ctx, arr), ctx)


def lbm_set_geometry(ctx, cell_type: np.ndarray):
    t = np.ascontiguousarray(cell_type, dtype=np.uint8)
    return _check(library().lbm_set_geometry(ctx, t.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))), ctx)


def lbm_set_fields(ctx, rho1: np.ndarray, rho2: np.ndarray, u: np.ndarray):
    r1 = np.ascontiguousarray(rho1, dtype=np.float64)
    r2 = np.ascontiguousarray(rho2, dtype=np.float64)
    uu = np.ascontiguousarray(u, dtype=np.float64)
    return _check(library().lbm_set_fields(ctx, _dp(r1), _dp(r2), _dp(uu)), ctx)


def lbm_step(ctx, n: int):
    return _check(library().lbm_step(ctx, int(n)), ctx)


def lbm_get_fields(ctx, rho1: np.ndarray, rho2: np.ndarray, u: np.ndarray):
    for a in (rho1, rho2, u):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return _check(library().lbm_get_fields(ctx, _dp(rho1), _dp(rho2), _dp(u)), ctx)


def lbm_reduce(ctx, out: np.ndarray, allow_diverged: bool = False):
    assert out.dtype == np.float64 and out.flags["C_CONTIGUOUS"]
    return _check(library().lbm_reduce(ctx, _dp(out)), ctx, allow=(4,) if allow_diverged else ())


def lbm_get_distributions(ctx, f: np.ndarray):
    assert f.dtype == np.float64 and f.flags["C_CONTIGUOUS"]
    return _check(library().lbm_get_distributions(ctx, _dp(f)), ctx)


def lbm_set_distributions(ctx, f: np.ndarray):
    a = np.ascontiguousarray(f, dtype=np.float64)
    return _check(library().lbm_set_distributions(ctx, _dp(a)), ctx)


def lbm_get_state(ctx) -> bytes:
    n = ctypes.c_size_t(0)
    _check(library().lbm_get_state(ctx, None, ctypes.byref(n)), ctx)
    buf = ctypes.create_string_buffer(n.value)
    _check(library().lbm_get_state(ctx, ctypes.cast(buf, ctypes.c_void_p), ctypes.byref(n)), ctx)
    return buf.raw[:n.value]


def lbm_set_state(ctx, state: bytes):
    buf = ctypes.create_string_buffer(state, len(state))
    return _check(library().lbm_set_state(ctx, ctypes.cast(buf, ctypes.c_void_p), len(state)), ctx)


def lbm_set_stream(ctx, stream_handle: int):
    return _check(library().lbm_set_stream(ctx, ctypes.c_void_p(int(stream_handle)) if stream_handle else None), ctx)


def lbm_set_barrier_test(ctx, wait_cycles: int, missing: int):
    return _check(library().lbm_set_barrier_test(ctx, int(wait_cycles), int(missing)), ctx)


def lbm_set_kernel(ctx, kernel):
    k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    return _check(library().lbm_set_kernel(ctx, k), ctx)


def lbm_set_tiling(ctx, tile: int, zchunk: int):
    return _check(library().lbm_set_tiling(ctx, int(tile), int(zchunk)), ctx)


def lbm_launch_count(ctx) -> int:
    return int(library().lbm_launch_count(ctx))


def lbm_resolved_kernel(ctx, n: int = 2) -> str:
    """Name of the strategy lbm_step(ctx, n) would run now."""
    L = library()
    L.lbm_resolved_kernel.argtypes = [ctypes.c_void_p, ctypes.c_int]
    k = int(L.lbm_resolved_kernel(ctx, int(n)))
    return {v: name for name, v in KERNELS.items()}.get(k, str(k))


PARTS = ("psi", "collide", "fused", "cluster")


def lbm_timing_begin(ctx, max_launches: int = 4096):
    L = library()
    L.lbm_timing_begin.argtypes = [ctypes.c_void_p, ctypes.c_int]
    return _check(L.lbm_timing_begin(ctx, int(max_launches)), ctx)


def lbm_timing_end(ctx) -> dict:
    """{part: (summed device ms, timed launches)} for the parts that ran."""
    L = library()
    L.lbm_timing_end.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
    ms = np.zeros(len(PARTS))
    n = (ctypes.c_longlong * len(PARTS))()
    _check(L.lbm_timing_end(ctx, _dp(ms), n), ctx)
    return {p: (float(ms[k]), int(n[k])) for k, p in enumerate(PARTS) if n[k] > 0}


def lbm_destroy(ctx):
    library().lbm_destroy(ctx)


class Sim:
    """Small convenience wrapper holding one context (same calls, same order)."""

    def __init__(self, nx, ny, nz, params, precision="fp64", eq_order=0, wall_model=2, kernel="auto", reg_order=2):
        self.shape = (len(params), nz, ny, nx)
        self.cfg = make_config(nx, ny, nz, len(params), precision, eq_order, wall_model, reg_order)
        self._params = make_params(params)
        self.ctx = lbm_create(self.cfg, self._params)
        if kernel != "auto":
            lbm_set_kernel(self.ctx, kernel)

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, cell_type):
        lbm_set_geometry(self.ctx, np.asarray(cell_type, dtype=np.uint8).reshape(self.shape))

    def set_params(self, params):
        if len(params) != self.shape[0]:
            raise ValueError("one parameter set per instance")
        lbm_set_params(self.ctx, params)

    def set_fields(self, rho1, rho2, u):
        lbm_set_fields(self.ctx, np.reshape(rho1, self.shape), np.reshape(rho2, self.shape),
                       np.reshape(u, self.shape + (3,)))

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def get_fields(self):
        r1 = np.zeros(self.shape)
        r2 = np.zeros(self.shape)
        u = np.zeros(self.shape + (3,))
        lbm_get_fields(self.ctx, r1, r2, u)
        return r1, r2, u

    def reduce(self, allow_diverged=False):
        out = np.zeros((self.shape[0], 7))
        lbm_reduce(self.ctx, out, allow_diverged)
        return out

    def get_f(self):
        out = np.zeros((self.shape[0], 2, 19) + self.shape[1:])
        lbm_get_distributions(self.ctx, out)
        return out

    def set_f(self, f):
        lbm_set_distributions(self.ctx, f)

    def get_state(self):
        return lbm_get_state(self.ctx)

    def set_state(self, s):
        lbm_set_state(self.ctx, s)

    @property
    def launches(self):
        return lbm_launch_count(self.ctx)


PLANE_PARTS = {"f_up": 0, "f_down": 1, "psi": 2}


def lbm_step_part(ctx, part: int):
    """Half of a split update: 0 the density pass, 1 the collision pass."""
    _check(library().lbm_step_part(ctx, int(part)), ctx)


def lbm_plane_bytes(ctx, what: str, z: int) -> int:
    n = ctypes.c_size_t(0)
    _check(library().lbm_plane_bytes(ctx, PLANE_PARTS[what], int(z), ctypes.byref(n)), ctx)
    return n.value


def lbm_plane_copy(ctx, what: str, z: int, buf_ptr: int, to_buf: bool):
    """Copy one plane's part between the context and the buffer at buf_ptr
    (host or device address, lbm_plane_bytes long)."""
    _check(library().lbm_plane_copy(ctx, PLANE_PARTS[what], int(z), buf_ptr, 1 if to_buf else 0), ctx)


def lbm_plane_get(ctx, what: str, z: int) -> np.ndarray:
    """One plane's crossing distributions or psi pairs as raw bytes (uint8)."""
    buf = np.empty(lbm_plane_bytes(ctx, what, z), dtype=np.uint8)
    if buf.size:
        lbm_plane_copy(ctx, what, z, buf.ctypes.data, True)
    return buf


def lbm_plane_set(ctx, what: str, z: int, buf: np.ndarray):
    b = np.ascontiguousarray(buf, dtype=np.uint8)
    if b.size != lbm_plane_bytes(ctx, what, z):
        raise ValueError("plane buffer has the wrong size")
    if b.size:
        lbm_plane_copy(ctx, what, z, b.ctypes.data, False)


def lbm_last_error(ctx=None) -> str:
    return library().lbm_last_error(ctx).decode()


def lbm_autotune(ctx, steps_per_trial: int = 5, cache_path: str | None = None):
    """Time the kernel strategies and tilings; returns (strategy, tile, zchunk)."""
    out = (ctypes.c_int * 3)()
    cp = cache_path.encode() if cache_path else None
    _check(library().lbm_autotune(ctx, int(steps_per_trial), cp, out), ctx)
    return tuple(out)


def lbm_run_to_steady(ctx, check_every: int, tol: float, max_steps: int, batch: int):
    """Advance until every residual <= tol; returns (updates done, residuals).
    Running out of max_steps (LBM_ERR_TIMEOUT) is not an error here: the
    caller sees it in the residuals."""
    done = ctypes.c_int(0)
    res = np.zeros(batch)
    rc = library().lbm_run_to_steady(ctx, int(check_every), float(tol), int(max_steps), ctypes.byref(done), _dp(res))
    _check(rc, ctx, allow=(5,))
    return done.value, res


def lbm_field_sums_static(rho1_ptr: int, rho2_ptr: int, u_ptr: int, type_ptr: int, ncells: int, batch: int,
                          out_ptr: int, stream: int = 0):
    """Mass and momentum sums of caller-owned device fields without any device
    allocation (raw device addresses, e.g. torch tensors' data_ptr()); writes
    out[batch][6] on the device.  For callers that must not allocate at this
    point: a fixed memory pool, a loop that cannot afford cudaMalloc's device
    synchronisation, or a host that owns all GPU memory."""
    L = library()
    f = L.lbm_field_sums_static
    f.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return _check(f(rho1_ptr, rho2_ptr, u_ptr, type_ptr, int(ncells), int(batch), out_ptr, stream or None))
