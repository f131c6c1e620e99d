"""FP64 CPU oracle of the two-component Shan-Chen D3Q19 update (arXiv:1711.03254).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, the smoke check and the
CPU-baseline leg of ``bench.py``.  The CUDA library never uses it and shares no
code with it.

The arithmetic lives in ``lbm_oracle.c`` (plain loops, FP64, no FMA
contraction); this module compiles it with gcc and exposes it through ctypes.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import shutil
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

Q = 19


def _compile(src: str, out: str) -> None:
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        _compile(_SRC, _LIB)
    return _LIB


class _Config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("batch", ctypes.c_int), ("eq_order", ctypes.c_int), ("wall_model", ctypes.c_int),
                ("reg_order", ctypes.c_int)]


class _Params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double * 2), ("G", ctypes.c_double), ("rho_s", ctypes.c_double),
                ("g", ctypes.c_double * 3), ("rho_in", ctypes.c_double * 2),
                ("u_in", ctypes.c_double * 3), ("slip", ctypes.c_double)]


def _load(path: str):
    L = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    vp = ctypes.c_void_p
    L.oracle_create.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_Params), ctypes.POINTER(vp)]
    L.oracle_destroy.argtypes = [vp]
    L.oracle_set_geometry.argtypes = [vp, ctypes.POINTER(ctypes.c_uint8)]
    L.oracle_set_fields.argtypes = [vp, dp, dp, dp]
    L.oracle_step.argtypes = [vp, ctypes.c_int]
    L.oracle_get_fields.argtypes = [vp, dp, dp, dp]
    L.oracle_get_f.argtypes = [vp, dp]
    L.oracle_set_f.argtypes = [vp, dp]
    L.oracle_reduce.argtypes = [vp, dp]
    L.oracle_get_force.argtypes = [vp, dp]
    L.oracle_step_count.argtypes = [vp]
    L.oracle_step_count.restype = ctypes.c_long
    L.oracle_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), dp, ctypes.POINTER(ctypes.c_int)]
    L.oracle_feq.argtypes = [ctypes.c_double, dp, ctypes.c_int, dp]
    L.oracle_pi_neq.argtypes = [dp, dp, dp]
    L.oracle_regularize.argtypes = [dp, dp]
    L.oracle_regularize3.argtypes = [dp, dp, dp]
    L.oracle_forcing.argtypes = [dp, dp, ctypes.c_double, ctypes.c_int, dp]
    L.oracle_tau_mix.argtypes = [ctypes.c_double, ctypes.c_double, dp]
    L.oracle_tau_mix.restype = ctypes.c_double
    L.oracle_collide_cell.argtypes = [dp, dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
    L.oracle_wall_potential.argtypes = [ctypes.c_double, dp]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _load(build())
    return _lib


@contextlib.contextmanager
def planted(old: str, new: str):
    """Mutation check for the pins: inside the block every function of this
    module runs an oracle compiled from a copy of lbm_oracle.c in which the
    text `old` (exactly one occurrence) is replaced by `new`.  A pin that still
    passes with a plausible slip planted this way cannot catch that slip."""
    global _lib
    text = open(_SRC).read()
    if text.count(old) != 1:
        raise ValueError(f"planted: {old!r} occurs {text.count(old)} times in the oracle source")
    d = tempfile.mkdtemp(prefix="oracle_planted_")
    try:
        src = os.path.join(d, "lbm_oracle_planted.c")
        with open(src, "w") as fh:
            fh.write(text.replace(old, new))
        so = os.path.join(d, "liboracle_planted.so")
        _compile(src, so)
        mutant = _load(so)
        with _lock:
            saved, _lib = _lib, mutant
        try:
            yield
        finally:
            with _lock:
                _lib = saved
    finally:
        shutil.rmtree(d, ignore_errors=True)


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --------------------------------------------------------------------------
# per-cell pieces (for the identity pins)
# --------------------------------------------------------------------------

def lattice():
    """D3Q19 velocities c [19,3] (int), weights w [19], opposite index [19]."""
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, dtype=np.int32)
    lib().oracle_lattice(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                         opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return c, w, opp


def feq(rho_a: float, u, eq_order: int = 0) -> np.ndarray:
    out = np.zeros(Q)
    lib().oracle_feq(float(rho_a), _dp(np.ascontiguousarray(u, dtype=np.float64)), int(eq_order), _dp(out))
    return out


def pi_neq(f, fe) -> np.ndarray:
    out = np.zeros(9)
    lib().oracle_pi_neq(_dp(np.ascontiguousarray(f, dtype=np.float64)),
                        _dp(np.ascontiguousarray(fe, dtype=np.float64)), _dp(out))
    return out.reshape(3, 3)


def regularize(pi) -> np.ndarray:
    out = np.zeros(Q)
    lib().oracle_regularize(_dp(np.ascontiguousarray(pi, dtype=np.float64).reshape(9)), _dp(out))
    return out


def regularize3(pi, u) -> np.ndarray:
    """f' of Eq. 10 with the third-order Hermite terms (recursive moments)."""
    out = np.zeros(Q)
    lib().oracle_regularize3(_dp(np.ascontiguousarray(pi, dtype=np.float64).reshape(9)),
                             _dp(np.ascontiguousarray(u, dtype=np.float64)), _dp(out))
    return out


def forcing(F, u, tau: float, eq_order: int = 0) -> np.ndarray:
    out = np.zeros(Q)
    lib().oracle_forcing(_dp(np.ascontiguousarray(F, dtype=np.float64)),
                         _dp(np.ascontiguousarray(u, dtype=np.float64)), float(tau), int(eq_order), _dp(out))
    return out


def tau_mix(rho1: float, rho2: float, tau) -> float:
    return lib().oracle_tau_mix(float(rho1), float(rho2), _dp(np.ascontiguousarray(tau, dtype=np.float64)))


def collide_cell(f, F, tau, eq_order: int = 0, reg_order: int = 2):
    """f [2,19] streamed, F [2,3] -> (f_post [2,19], u_F [3], rho [2], tau_mix)."""
    fo = np.zeros(2 * Q)
    uF = np.zeros(3)
    r = np.zeros(2)
    tm = np.zeros(1)
    lib().oracle_collide_cell(_dp(np.ascontiguousarray(f, dtype=np.float64).reshape(-1)),
                              _dp(np.ascontiguousarray(F, dtype=np.float64).reshape(-1)),
                              _dp(np.ascontiguousarray(tau, dtype=np.float64)), int(eq_order), int(reg_order),
                              _dp(fo), _dp(uF), _dp(r), _dp(tm))
    return fo.reshape(2, Q), uF, r, float(tm[0])


def wall_potential(rho_s: float) -> np.ndarray:
    out = np.zeros(2)
    lib().oracle_wall_potential(float(rho_s), _dp(out))
    return out


# --------------------------------------------------------------------------
# domain
# --------------------------------------------------------------------------

class OracleSim:
    """Whole-domain oracle; same call shape as the CUDA binding.

    params: list (length batch) of dicts with keys tau (2), G, rho_s, g (3),
    rho_in (2), u_in (3).  Fields are numpy float64 arrays shaped
    [batch, nz, ny, nx] (u: [batch, nz, ny, nx, 3]).
    """

    def __init__(self, nx, ny, nz, params, eq_order=0, wall_model=2, reg_order=2):
        self.shape = (len(params), nz, ny, nx)
        cfg = _Config(nx, ny, nz, len(params), eq_order, wall_model, reg_order)
        arr = (_Params * len(params))()
        for k, p in enumerate(params):
            arr[k].tau[:] = list(p.get("tau", (1.0, 1.0)))
            arr[k].G = p.get("G", 0.0)
            arr[k].rho_s = p.get("rho_s", 0.0)
            arr[k].g[:] = list(p.get("g", (0.0, 0.0, 0.0)))
            arr[k].rho_in[:] = list(p.get("rho_in", (0.0, 0.0)))
            arr[k].u_in[:] = list(p.get("u_in", (0.0, 0.0, 0.0)))
            arr[k].slip = p.get("slip", 0.0)
        h = ctypes.c_void_p()
        rc = lib().oracle_create(ctypes.byref(cfg), arr, ctypes.byref(h))
        if rc != 0:
            raise ValueError("oracle_create rejected the configuration")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def set_geometry(self, cell_type: np.ndarray):
        t = np.ascontiguousarray(cell_type, dtype=np.uint8).reshape(self.shape)
        if lib().oracle_set_geometry(self._h, t.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))) != 0:
            raise ValueError("bad cell type")

    def set_fields(self, rho1, rho2, u):
        r1 = np.ascontiguousarray(rho1, dtype=np.float64).reshape(self.shape)
        r2 = np.ascontiguousarray(rho2, dtype=np.float64).reshape(self.shape)
        uu = np.ascontiguousarray(u, dtype=np.float64).reshape(self.shape + (3,))
        lib().oracle_set_fields(self._h, _dp(r1), _dp(r2), _dp(uu))

    def step(self, n: int = 1):
        if lib().oracle_step(self._h, int(n)) != 0:
            raise ValueError("bad step count")

    def get_fields(self):
        r1 = np.zeros(self.shape)
        r2 = np.zeros(self.shape)
        u = np.zeros(self.shape + (3,))
        lib().oracle_get_fields(self._h, _dp(r1), _dp(r2), _dp(u))
        return r1, r2, u

    def get_f(self):
        out = np.zeros((self.shape[0], 2, Q) + self.shape[1:])
        lib().oracle_get_f(self._h, _dp(out))
        return out

    def set_f(self, f):
        a = np.ascontiguousarray(f, dtype=np.float64)
        lib().oracle_set_f(self._h, _dp(a))

    def get_force(self):
        """Total force per component of the last update, [batch, 2, nz, ny, nx, 3]."""
        out = np.zeros((self.shape[0], 2) + self.shape[1:] + (3,))
        lib().oracle_get_force(self._h, _dp(out))
        return out

    def reduce(self):
        out = np.zeros((self.shape[0], 7))
        lib().oracle_reduce(self._h, _dp(out))
        return out

    @property
    def step_count(self) -> int:
        return int(lib().oracle_step_count(self._h))
